// rti_instantiate.cuh -- launchers for one precision RTI_T (included once per .cu).
#include "rti_kernels.cuh"
#include "rti_launch.h"

namespace rti {

namespace {
// the step kernel of variant `mode` (kStepPlain or kStepTrack, plus kStepLimit and
// kStepFull; the full-feedback variants are k_step_flow)
using StepFn = void (*)(KParams<RTI_T>, int, int);
StepFn step_kernel(int mode) {
  switch (mode) {
    case 0: return k_step<RTI_T, 0>;
    case 1: return k_step<RTI_T, 1>;
    case 2: return k_step<RTI_T, 2>;
    case 3: return k_step<RTI_T, 3>;
    case 4: return k_step_flow<RTI_T, 4>;
    case 5: return k_step_flow<RTI_T, 5>;
    case 6: return k_step_flow<RTI_T, 6>;
    case 7: return k_step_flow<RTI_T, 7>;
    default: return nullptr;
  }
}
}  // namespace

template <>
cudaError_t persistent_grid<RTI_T>(int* grid, int tx, int ty, int mode, int cap) {
  (void)tx;
  (void)ty;
  const StepFn fn = step_kernel(mode);
  if (!fn) return cudaErrorInvalidValue;
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kWarps * 32, 0);
  if (e == cudaSuccess && cap > 0 && per > cap) per = cap;
  if (e == cudaSuccess) *grid = sms * (per > 0 ? per : 1);
  return e;
}

template <>
cudaError_t launch_chunk<RTI_T>(const KParams<RTI_T>& kp, int schedule, int grid,
                                const int* nscen, cudaStream_t st) {
  const dim3 blk(32, kWarps);
  const int mode = (kp.track ? kStepTrack : kStepPlain) | (kp.limit ? kStepLimit : 0) |
                   (kp.full ? kStepFull : 0);
  cudaError_t e = cudaMemsetAsync(kp.bar, 0, sizeof(Bar), st);  // barrier and strip counters
  if (e == cudaSuccess && kp.full)  // the strip flags of full feedback
    e = cudaMemsetAsync(kp.done, 0, (size_t)kp.ndone * sizeof(*kp.done), st);
  if (e != cudaSuccess) return e;
  if (schedule == 0) {  // one cooperative launch for the whole chunk
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = blk;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, step_kernel(mode), kp, 0, kp.nsteps);
  } else {  // one launch per step
    const StepFn fn = step_kernel(mode);
    for (int s = 0; s < kp.nsteps && e == cudaSuccess; ++s) {
      fn<<<grid, blk, 0, st>>>(kp, s, 1);
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) return e;
  k_advance<<<1, 256, 0, st>>>(kp.scen, nscen, kp.nsteps);
  return cudaGetLastError();
}

template <>
cudaError_t launch_snapshot<RTI_T>(const KParams<RTI_T>& kp, int grid, cudaStream_t st) {
  k_snapshot<RTI_T><<<grid, dim3(32, 8), 0, st>>>(kp);
  return cudaGetLastError();
}

template <>
cudaError_t launch_fill_edges<RTI_T>(const KParams<RTI_T>& kp, int grid, int parity,
                                     cudaStream_t st) {
  k_fill_edges<RTI_T><<<grid, dim3(32, 8), 0, st>>>(kp, parity);
  return cudaGetLastError();
}

}  // namespace rti
