// Column kernels of the small geometries (N = 2^12 and 2^8), every launch shape.
#include "cols.cuh"

namespace ckks {

#define CKKS_COL_INST(G)                                                                                        \
  template void launch_modup_cols<G>(const DevParams&, int, int, int, int, const Scratch&, const ColShape&,     \
                                     cudaStream_t);                                                           \
  template void launch_moddown_cols<G>(const DevParams&, int, int, int, const Scratch&, const ColShape&, cudaStream_t); \
  template void launch_rs_cols_fused<G>(const DevParams&, int, const Scratch&, uint32_t*, const ColShape&,       \
                                        cudaStream_t);                                                        \
  template void launch_mm_cols<G>(const DevParams&, const MmArgs&, const Scratch&, const ColShape&, cudaStream_t);
using G12 = Geo<8, 8>;
using G8 = Geo<4, 4>;
CKKS_COL_INST(G12)
CKKS_COL_INST(G8)
#undef CKKS_COL_INST

}  // namespace ckks
