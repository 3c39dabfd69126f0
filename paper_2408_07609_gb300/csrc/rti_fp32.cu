// Binary32 kernels (eta stored as the deviation from still water).
#define RTI_T float
#include "rti_instantiate.cuh"

namespace rti {
__global__ void k_advance(ScenDev* sc, const int* nscen, int nsteps) {
  const int n = *nscen;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    long long d = sc[k].remaining < nsteps ? sc[k].remaining : nsteps;
    if (d < 0) d = 0;
    sc[k].base += d;
    sc[k].remaining -= d;
  }
}
}  // namespace rti

namespace rti {
__global__ void k_set_scen(ScenDev* sc, int idx, long long base, long long remaining) {
  sc[idx].base = base;
  sc[idx].remaining = remaining;
}
}  // namespace rti

#ifdef RTI_CHECKED
namespace rti {
cudaError_t debug_check_fp32(int* out8) {
  return cudaMemcpyFromSymbol(out8, g_rti_check, 8 * sizeof(int));
}
}  // namespace rti
#endif
