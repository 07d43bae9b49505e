// Fused and merged ModDown + rescale column kernels at N = 2^16, every launch shape.
#include "cols.cuh"

namespace ckks {

template void launch_rs_cols_fused<Geo<8, 32>>(const DevParams&, int, const Scratch&, uint32_t*, const ColShape&,
                                               cudaStream_t);
template void launch_mm_cols<Geo<8, 32>>(const DevParams&, const MmArgs&, const Scratch&, const ColShape&,
                                         cudaStream_t);

}  // namespace ckks
