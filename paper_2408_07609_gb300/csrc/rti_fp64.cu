// Binary64 kernels. Built with -fmad=false: no multiply-add is fused, so every
// operation rounds exactly as in the FP64 oracle's source order.
#define RTI_T double
#include "rti_instantiate.cuh"

#ifdef RTI_CHECKED
namespace rti {
cudaError_t debug_check_fp64(int* out8) {
  return cudaMemcpyFromSymbol(out8, g_rti_check, 8 * sizeof(int));
}
}  // namespace rti
#endif
