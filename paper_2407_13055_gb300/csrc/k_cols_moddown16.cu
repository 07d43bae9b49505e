// ModDown column kernels at N = 2^16, every launch shape.
#include "cols.cuh"

namespace ckks {

template void launch_moddown_cols<Geo<8, 32>>(const DevParams&, int, int, int, const Scratch&, const ColShape&, cudaStream_t);

}  // namespace ckks
