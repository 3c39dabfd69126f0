// rti_kernels.cuh -- sm_103a kernels of the nested TUNAMI-N2 leap-frog step.
//
// Included by rti_fp32.cu and rti_fp64.cu, which instantiate it for binary32 and
// binary64 state. One time step is two passes over a tile work list that holds the
// tiles of every block of every scenario in a batch:
//
//   pass A (Eq. 1, Sec. IV-A "NLMASS"): eta^{n+1} = eta^n - dt/dx (dM + dN), the dry
//     clip, the coarse-to-fine edge fluxes of a child (pulled from the parent's
//     current fluxes and stored into the child's flux array), the fine-to-coarse
//     ring of a parent (Listing 5 mean of the 3x3 child cells, recomputed from the
//     child's stable time level), max height / arrival (output update) and the
//     per-tile binary64 volume budget (warp-shuffle reduction);
//   pass B (Eqs. 2-3, "NLMNT2"/XMMT/YMMT): M^{n+1}, N^{n+1} with upwind advection,
//     pressure on the total depth, semi-implicit Manning friction, the wet/dry front
//     and the outflow limit; radiation or wall faces on root edges. A tile stages its
//     fields with a two-cell halo in shared memory, computes every face's advective
//     fluxes once, then updates its faces from shared memory.
//
// eta, M and N are ping-ponged (parity = step & 1), so no pass reads what it writes
// and every pull reads a time level that no tile of the same pass modifies.
// The discrete rules follow the oracle's readings R1-R10 operation for operation;
// the binary64 build uses -fmad=false so that it rounds like the oracle.
//
// Block descriptors: a tile copies its block's descriptor (and, for a child, its
// parent's) into shared memory once and reads fields from there. Optimised binary64
// builds that re-read descriptor fields through references into the device table
// faulted on an in-range edge read (the range-checked, -G and copied-descriptor builds
// did not); the mixed-sequence GPU test guards this.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rti_layout.h"

namespace rti {

__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dcbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float dcbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ bool dfinite(double x) { return isfinite(x); }
__device__ __forceinline__ bool dfinite(float x) { return isfinite(x); }

#ifdef RTI_CHECKED
// Checked build: every array index is tested against the pitched allocation. The first
// bad one is recorded in g_rti_check (code, column, row, extent) and the access is
// redirected to element 0 of the array, which lies in the margin.
static __device__ int g_rti_check[8];  // one copy per module (binary32 and binary64)
__device__ __forceinline__ size_t checked_ix(int c, int r, int pitch, int ny, int code) {
  if (c < -kXOff || c + kXOff >= pitch || r < -kYOff || r > ny + kYOff) {
    if (atomicCAS(&g_rti_check[0], 0, code) == 0) {
      g_rti_check[1] = c;
      g_rti_check[2] = r;
      g_rti_check[3] = pitch;
      g_rti_check[4] = ny;
      g_rti_check[5] = blockIdx.x;
    }
    return 0;
  }
  return (size_t)(r + kYOff) * (size_t)pitch + (size_t)(c + kXOff);
}
__device__ __forceinline__ int checked_idx(int i, int n, int code) {
  if (i < 0 || i >= n) {
    if (atomicCAS(&g_rti_check[0], 0, code) == 0) {
      g_rti_check[1] = i;
      g_rti_check[2] = n;
      g_rti_check[5] = blockIdx.x;
    }
    return 0;
  }
  return i;
}
#define RTI_IX(c, r, pitch, ny, code) checked_ix((c), (r), (pitch), (ny), (code))
#define RTI_BLK(kp, i) (kp).blk[checked_idx((i), (kp).nblk, 10)]
#define RTI_KID(kp, i) (kp).kids[checked_idx((i), (kp).nkids, 11)]
#else
#define RTI_IX(c, r, pitch, ny, code) ((size_t)((r) + kYOff) * (size_t)(pitch) + (size_t)((c) + kXOff))
#define RTI_BLK(kp, i) (kp).blk[(i)]
#define RTI_KID(kp, i) (kp).kids[(i)]
#endif

template <class T>
__device__ __forceinline__ size_t ix(const Blk<T>& b, int c, int r) {
  return RTI_IX(c, r, b.pitch, b.ny, 1);
}

// Copy a descriptor from the device table into shared memory (all threads call it;
// the caller synchronises before use).
template <class T>
__device__ __forceinline__ void stage_blk(Blk<T>* dst, const Blk<T>* src) {
  static_assert(sizeof(Blk<T>) % 4 == 0, "descriptor size");
  const int tid = threadIdx.x + 32 * threadIdx.y;
  const unsigned* s = reinterpret_cast<const unsigned*>(src);
  unsigned* d = reinterpret_cast<unsigned*>(dst);
  for (int w = tid; w < (int)(sizeof(Blk<T>) / 4); w += 256) d[w] = s[w];
}

// ------------------------------------------------------------------ coarse -> fine (R7)
// Fine face t of an edge whose coarse faces are v(k), k = 0..K-1: the coarse value at
// the middle fine face, (2 v_k + v_{k+-1}) / 3 at the outer ones, neighbour clamped.
template <class T>
__device__ __noinline__ T edge_interp(const T* arr, const Blk<T>& P, int fixed, int start, int K,
                                      int t, bool along_y) {
  int k = t / 3, sub = t - 3 * k;
  double vk = along_y ? (double)arr[ix(P, fixed, start + k)] : (double)arr[ix(P, start + k, fixed)];
  if (sub == 1) return (T)vk;
  int kn = sub == 0 ? k - 1 : k + 1;
  kn = kn < 0 ? 0 : (kn > K - 1 ? K - 1 : kn);
  double vn = along_y ? (double)arr[ix(P, fixed, start + kn)] : (double)arr[ix(P, start + kn, fixed)];
  return (T)((2.0 * vk + vn) / 3.0);
}

// x-flux of face (f, j) at parity p; a child's edge faces come from its parent P.
template <class T>
__device__ __forceinline__ T face_m(const Blk<T>& b, const Blk<T>& P, int p, int f, int j) {
  if (b.is_child && (f == 0 || f == b.nx)) {
    int F = b.i0 + (f == 0 ? 0 : b.nx / 3);
    return edge_interp<T>(P.M[p], P, F, b.j0, b.ny / 3, j, true);
  }
  return b.M[p][ix(b, f, j)];
}
template <class T>
__device__ __forceinline__ T face_n(const Blk<T>& b, const Blk<T>& P, int p, int i, int g) {
  if (b.is_child && (g == 0 || g == b.ny)) {
    int G = b.j0 + (g == 0 ? 0 : b.ny / 3);
    return edge_interp<T>(P.N[p], P, G, b.i0, b.nx / 3, i, false);
  }
  return b.N[p][ix(b, i, g)];
}

// ------------------------------------------------------------------ mass (R1 + R5)
template <class T>
__device__ __forceinline__ T mass(const Blk<T>& b, int p, int i, int j, T Mw, T Me, T Ns, T Nn,
                                  double& clip) {
  size_t c = ix(b, i, j);
  T h = b.h[c];
  T e = b.eta[p][c] - (b.dtdx * (Me - Mw) + b.dtdx * (Nn - Ns));
  if (h + e < T(0)) {
    clip += (double)(-h - e) * b.dx2;
    e = -h;
  }
  return e;
}

// eta^{n+1} of child cell (x, y) recomputed from the child's stable level p; P is the
// child's parent (the block whose ring is being filled).
template <class T>
__device__ T child_eta_next(const Blk<T>& c, const Blk<T>& P, int p, int x, int y) {
  T Mw = face_m(c, P, p, x, y), Me = face_m(c, P, p, x + 1, y);
  T Ns = face_n(c, P, p, x, y), Nn = face_n(c, P, p, x, y + 1);
  double dummy = 0.0;
  return mass(c, p, x, y, Mw, Me, Ns, Nn, dummy);
}

// ------------------------------------------------------------------ fine -> coarse (R8)
// If parent cell (I, J) of block b lies on the inner ring of a child footprint and the
// 3x3 patch has a wet cell, store the floored mean of the wet child levels in `out`.
template <class T>
__device__ __noinline__ bool ring_value(const KParams<T>& kp, const Blk<T>& b, int p, int I,
                                        int J, T hP, T& out) {
  for (int q = 0; q < b.child_count; ++q) {
    const Blk<T> c = RTI_BLK(kp, RTI_KID(kp, b.child_first + q));
    int a = c.nx / 3, bb = c.ny / 3;
    int u = I - c.i0, v = J - c.j0;
    if (u < 0 || v < 0 || u >= a || v >= bb) continue;
    if (!(u == 0 || u == a - 1 || v == 0 || v == bb - 1)) return false;
    double sum = 0.0;
    int wet = 0;
    for (int x = 3 * u; x < 3 * u + 3; ++x) {    // outer: x (the paper's J)
      for (int y = 3 * v; y < 3 * v + 3; ++y) {  // inner: y (the paper's I)
        T e = child_eta_next(c, b, p, x, y);
        if (c.h[ix(c, x, y)] + e > c.eps) {
          sum = sum + (double)e;
          wet = wet + 1;
        }
      }
    }
    if (wet == 0) return false;
    double avg = sum * (1.0 / (double)wet);
    if (avg < -(double)hP) avg = -(double)hP;
    out = (T)avg;
    return true;
  }
  return false;
}

// ------------------------------------------------------------------ momentum (R2-R4, R6)
template <class T>
__device__ __forceinline__ T upwind(T w, T phim, T phi0, T phip, bool okm, bool okp) {
  if (w > T(0)) return okm ? phi0 - phim : T(0);
  if (w < T(0)) return okp ? phip - phi0 : T(0);
  return (okm && okp) ? T(0.5) * (phip - phim) : T(0);
}

// Arithmetic of the momentum update in the state precision. Binary64 keeps the oracle's
// exact expressions (correctly rounded divide and square root, library cbrt) so that it
// reproduces the oracle's rounding. Binary32 (the forecast path, checked against the
// oracle within the stated accuracy) uses the special-function unit: approximate
// reciprocal, reciprocal square root, and D^(-7/3) = exp(-7/3 ln D).
template <class T>
struct Ar;
template <>
struct Ar<double> {
  static __device__ __forceinline__ double quot(double a, double b) { return a / b; }
  static __device__ __forceinline__ double update(double m, double across, double Df,
                                                  double grad, double adv, double nf,
                                                  double g, double dtdx, double cfric) {
    double P = g * Df * dtdx * grad;
    double F = cfric * nf * nf * sqrt(m * m + across * across) / (Df * Df * cbrt(Df));
    return ((1.0 - F) * m - adv - P) / (1.0 + F);
  }
};
template <>
struct Ar<float> {
  static __device__ __forceinline__ float quot(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float update(float m, float across, float Df, float grad,
                                                 float adv, float nf, float g, float dtdx,
                                                 float cfric) {
    const float P = g * Df * dtdx * grad;
    const float s2 = m * m + across * across;
    const float sq = s2 > 0.0f ? s2 * rsqrtf(s2) : 0.0f;
    const float d73inv = __expf(-2.33333333f * __logf(Df));
    const float F = cfric * nf * nf * sq * d73inv;
    return __fdividef((1.0f - F) * m - adv - P, 1.0f + F);
  }
};

template <class T>
__device__ __forceinline__ T flux_update(const Blk<T>& b, T m, T across, T Df, T grad, T adv,
                                         T nf) {
  return Ar<T>::update(m, across, Df, grad, adv, nf, b.g, b.dtdx, b.cfric);
}

template <class T>
__device__ __forceinline__ T limit_outflow(T m, T Dlo, T Dhi, T dx, T q4dt) {
  T cap = (m > T(0) ? Dlo : Dhi) * dx / q4dt;
  if (m > cap) return cap;
  if (m < -cap) return -cap;
  return m;
}

// Shared-memory tile of pass B. Local point (lx, ly) holds cell, x-face and y-face
// (x0 - 2 + lx, y0 - 2 + ly) of the block; W = tx + 4 columns, ty + 4 rows.
//   E, H, NM, MX, NY : eta^{n+1}, h, Manning n, M^n, N^n (loaded, zero off the margins)
//   QX, RX, VX       : M^2/D, M Nbar/D and "usable by advection" of x-faces
//   SY, TY, VY       : N^2/D, N Mbar/D and "usable by advection" of y-faces
template <class T>
struct BTile {
  T *E, *H, *MX, *NY, *QX, *RX, *SY, *TY;
  float* NM;
  unsigned char *VX, *VY;
  int W;
};

__host__ __device__ __forceinline__ size_t btile_bytes(int tx, int ty, size_t elem) {
  const size_t P = (size_t)(tx + 4) * (size_t)(ty + 4);
  return (P * (8 * elem + 4 + 2) + 15) / 16 * 16;
}

template <class T>
__device__ __forceinline__ BTile<T> carve_btile(unsigned char* base, int tx, int ty) {
  BTile<T> S;
  S.W = tx + 4;
  const int P = (tx + 4) * (ty + 4);
  T* t = reinterpret_cast<T*>(base);
  S.E = t;
  S.H = t + P;
  S.MX = t + 2 * P;
  S.NY = t + 3 * P;
  S.QX = t + 4 * P;
  S.RX = t + 5 * P;
  S.SY = t + 6 * P;
  S.TY = t + 7 * P;
  S.NM = reinterpret_cast<float*>(t + 8 * P);
  S.VX = reinterpret_cast<unsigned char*>(S.NM + P);
  S.VY = S.VX + P;
  return S;
}

// R2 + R4 at interior x-face (f, j); k = local index of cell (f, j)
template <class T>
__device__ __forceinline__ T xmom_s(const Blk<T>& b, const BTile<T>& S, int k) {
  const T eps = b.eps;
  const int W = S.W;
  const T eL = S.E[k - 1], eR = S.E[k], hL = S.H[k - 1], hR = S.H[k];
  const bool wL = hL + eL > eps, wR = hR + eR > eps;
  const T m = S.MX[k];
  const T nb = T(0.25) * ((S.NY[k - 1] + S.NY[k]) + (S.NY[k - 1 + W] + S.NY[k + W]));
  T Df, grad, adv;
  if (wL && wR) {
    Df = T(0.5) * (hL + hR) + T(0.5) * (eL + eR);
    grad = eR - eL;
    const bool okm = S.VX[k - 1], okp = S.VX[k + 1];
    const T ax = upwind(m, okm ? S.QX[k - 1] : T(0), S.QX[k], okp ? S.QX[k + 1] : T(0), okm, okp);
    const bool oks = S.VX[k - W], okn = S.VX[k + W];
    const T ay = upwind(nb, oks ? S.RX[k - W] : T(0), S.RX[k], okn ? S.RX[k + W] : T(0), oks, okn);
    adv = b.dtdx * (ax + ay);
  } else if (wL && !wR && eL > -hR) {
    Df = eL + hR;
    grad = -hR - eL;
    adv = T(0);
  } else if (wR && !wL && eR > -hL) {
    Df = eR + hL;
    grad = eR + hL;
    adv = T(0);
  } else {
    return T(0);
  }
  if (!(Df > eps)) return T(0);
  const float nL = S.NM[k - 1], nR = S.NM[k];
  const T nf = (T)(nL > nR ? nL : nR);
  const T m1 = flux_update(b, m, nb, Df, grad, adv, nf);
  if (!(wL && wR) && (wL ? m1 < T(0) : m1 > T(0))) return T(0);
  return limit_outflow(m1, hL + eL, hR + eR, b.dx, b.q4dt);
}

// R3 + R4 at interior y-face (i, g); k = local index of cell (i, g)
template <class T>
__device__ __forceinline__ T ymom_s(const Blk<T>& b, const BTile<T>& S, int k) {
  const T eps = b.eps;
  const int W = S.W;
  const T eS = S.E[k - W], eN = S.E[k], hS = S.H[k - W], hN = S.H[k];
  const bool wS = hS + eS > eps, wN = hN + eN > eps;
  const T v = S.NY[k];
  const T mb = T(0.25) * ((S.MX[k - W] + S.MX[k]) + (S.MX[k - W + 1] + S.MX[k + 1]));
  T Df, grad, adv;
  if (wS && wN) {
    Df = T(0.5) * (hS + hN) + T(0.5) * (eS + eN);
    grad = eN - eS;
    const bool okm = S.VY[k - W], okp = S.VY[k + W];
    const T ay = upwind(v, okm ? S.SY[k - W] : T(0), S.SY[k], okp ? S.SY[k + W] : T(0), okm, okp);
    const bool okw = S.VY[k - 1], oke = S.VY[k + 1];
    const T ax = upwind(mb, okw ? S.TY[k - 1] : T(0), S.TY[k], oke ? S.TY[k + 1] : T(0), okw, oke);
    adv = b.dtdx * (ay + ax);
  } else if (wS && !wN && eS > -hN) {
    Df = eS + hN;
    grad = -hN - eS;
    adv = T(0);
  } else if (wN && !wS && eN > -hS) {
    Df = eN + hS;
    grad = eN + hS;
    adv = T(0);
  } else {
    return T(0);
  }
  if (!(Df > eps)) return T(0);
  const float nS = S.NM[k - W], nN = S.NM[k];
  const T nf = (T)(nS > nN ? nS : nN);
  const T v1 = flux_update(b, v, mb, Df, grad, adv, nf);
  if (!(wS && wN) && (wS ? v1 < T(0) : v1 > T(0))) return T(0);
  return limit_outflow(v1, hS + eS, hN + eN, b.dx, b.q4dt);
}

// R6: flux leaving through a root edge next to cell k (sign +1 east/north, -1 west/south)
template <class T>
__device__ __forceinline__ T radiate_s(const Blk<T>& b, const BTile<T>& S, int k, T sign) {
  const T h = S.H[k], e = S.E[k];
  if (!(h + e > b.eps)) return T(0);
  return sign * (dsqrt(b.g * (h > T(0) ? h : T(0))) * e);
}

// ------------------------------------------------------------------ block reduction
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ async copy pipeline
// A CTA walks its tiles of one pass with two shared-memory stages: warp 0 issues the
// bulk copies (cp.async.bulk, one per row segment of each field) of the next tile into
// one stage while all warps compute the tile held in the other. Each stage has an
// mbarrier that completes when the copies have landed (transaction count) and warp 0
// has arrived; every wait on it is bounded.

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false after `limit` cycles (the caller records a timeout).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}
// One bulk copy global -> shared of `bytes` (both 16-byte aligned, bytes % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Generic-proxy accesses before this point are ordered before later async-proxy ones.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async;" ::: "memory");
}

// Shared-memory layout of the pipeline (host and device agree on it).
struct PipeLayout {
  int SW, SH;          // stage row width (elements) and rows
  size_t hdr, stage, derived, total;
};
template <class T>
struct SlotHdr {       // what the issuing warp records for the tile in a stage
  Blk<T> b;            // the tile's block descriptor
  Blk<T> P;            // its parent's (children only)
  Tile td;
  int p, sn, active;
};
// The issuing warp's cache of the last block it staged (tiles of a CTA mostly come
// from the same block): descriptors and the scenario counters of this chunk.
template <class T>
struct IssueCache {
  Blk<T> b;
  Blk<T> P;
  ScenDev sc;
  int blk;  // block index of the cached entry, -1 when empty
};
template <class T>
__host__ __device__ __forceinline__ PipeLayout pipe_layout(int tx, int ty) {
  PipeLayout L;
  L.SW = tx + 8;
  L.SH = ty + 4;
  const size_t n = (size_t)L.SW * L.SH;
  L.hdr = (2 * sizeof(unsigned long long) + 2 * sizeof(SlotHdr<T>) + sizeof(IssueCache<T>) +
           127) / 128 * 128;
  // pass B: eta^{n+1}, h, M, N (T) and Manning n (float); pass A needs less
  L.stage = (n * (4 * sizeof(T) + sizeof(float)) + 127) / 128 * 128;
  // pass B's face terms QX, RX, SY, TY (T) and the two validity byte arrays
  L.derived = (n * (4 * sizeof(T) + 2) + 127) / 128 * 128;
  L.total = L.hdr + 2 * L.stage + L.derived;
  return L;
}

struct PipeState {
  unsigned phase;  // bit s: parity of stage s's next completion
};

// Static shared memory of the step kernels.
struct StepShared {
  double red[4][8];
  int go;
  int fail;
};

// Warp 0: record tile t in slot H and issue the copies of the rows pass A (passB false)
// or pass B (passB true) reads into `stage`, completing on `bar`.
//   pass A rows y0..ye-1 (N one more), columns [x0, x0 + tx + 4): eta^n, M^n, N^n, h, max
//   pass B rows y0-2..ye+1, columns [x0 - 4, x0 + tx + 4): eta^{n+1}, h, M^n, N^n, n
// Column ends are clamped to the allocated row (pitch - 4), row ends to ny + 2; every
// segment starts on a 16-byte boundary (x0 is a multiple of the 32-wide tile).
template <class T>
__device__ __forceinline__ void warp_copy(void* dst, const void* src, int bytes) {
  const unsigned* s = reinterpret_cast<const unsigned*>(src);
  unsigned* d = reinterpret_cast<unsigned*>(dst);
  for (int w = threadIdx.x; w < bytes / 4; w += 32) d[w] = s[w];
}

template <class T>
__device__ void issue_tile(const KParams<T>& kp, int t, int s, bool passB, SlotHdr<T>& H,
                           IssueCache<T>& cache, unsigned char* stage, unsigned long long* bar,
                           const PipeLayout& L) {
  const int lane = threadIdx.x;
  const Tile td = kp.tiles[t];
  if (td.blk != cache.blk) {  // new block: descriptors and counters from the device tables
    warp_copy<T>(&cache.b, &RTI_BLK(kp, td.blk), sizeof(Blk<T>));
    __syncwarp();
    if (cache.b.is_child) warp_copy<T>(&cache.P, &RTI_BLK(kp, cache.b.parent), sizeof(Blk<T>));
    if (lane == 0) {
      cache.sc = kp.scen[cache.b.scen];
      cache.blk = td.blk;
    }
    __syncwarp();
  }
  warp_copy<T>(&H.b, &cache.b, sizeof(Blk<T>));
  if (cache.b.is_child && !passB) warp_copy<T>(&H.P, &cache.P, sizeof(Blk<T>));
  __syncwarp();
  const ScenDev sc = cache.sc;
  const bool active = (long long)s < sc.remaining;
  const int p = (int)((sc.base + s) & 1);
  const Blk<T>& b = H.b;
  const int x0 = td.x0, y0 = td.y0;
  const int ye = min(y0 + kp.ty, b.ny);
  const int cbeg = passB ? x0 - 4 : x0;
  const int cend = min(x0 + kp.tx + 4, b.pitch - kXOff);
  const int ncol = cend - cbeg;
  const int rbeg = passB ? y0 - 2 : y0;
  const int nrow = passB ? min(ye + 2, b.ny + 3) - rbeg : ye - y0;
  const int SW = L.SW;
  // field list: (source array, element size, shared offset in bytes, rows)
  const T* src[5];
  size_t off[5];
  int rows[5], esz[5];
  const size_t plane = (size_t)SW * L.SH;
  if (!passB) {
    src[0] = b.eta[p]; src[1] = b.M[p]; src[2] = b.N[p]; src[3] = b.h; src[4] = b.emax;
    const size_t ty1 = (size_t)SW * kp.ty * sizeof(T);
    off[0] = 0; off[1] = ty1; off[2] = 2 * ty1; off[3] = 3 * ty1 + SW * sizeof(T);
    off[4] = 4 * ty1 + SW * sizeof(T);
    rows[0] = rows[1] = rows[3] = rows[4] = nrow;
    rows[2] = nrow + 1;
    esz[0] = esz[1] = esz[2] = esz[3] = esz[4] = sizeof(T);
  } else {
    src[0] = b.eta[p ^ 1]; src[1] = b.h; src[2] = b.M[p]; src[3] = b.N[p];
    src[4] = reinterpret_cast<const T*>(b.man);
    for (int f = 0; f < 4; ++f) off[f] = f * plane * sizeof(T);
    off[4] = 4 * plane * sizeof(T);
    for (int f = 0; f < 5; ++f) rows[f] = nrow;
    esz[0] = esz[1] = esz[2] = esz[3] = sizeof(T);
    esz[4] = sizeof(float);
  }
  unsigned total = 0;
  for (int f = 0; f < 5; ++f) total += (unsigned)(rows[f] * ncol * esz[f]);
  if (lane == 0) {
    H.td = td;
    H.p = p;
    H.sn = (int)(sc.base + s + 1);
    H.active = active;
    mbar_arrive_tx(bar, active ? total : 0u);
  }
  __syncwarp();
  if (!active) return;
  int ncopy = 0;
  for (int f = 0; f < 5; ++f) ncopy += rows[f];
  for (int k = lane; k < ncopy; k += 32) {
    int f = 0, r = k;
    while (r >= rows[f]) r -= rows[f++];
    const int gr = rbeg + r;
    const char* g = reinterpret_cast<const char*>(src[f]) +
                    ((size_t)(gr + kYOff) * b.pitch + (size_t)(cbeg + kXOff)) * esz[f];
    unsigned char* d = stage + off[f] + (size_t)r * SW * esz[f];
    bulk_g2s(d, g, (unsigned)(ncol * esz[f]), bar);
  }
}

// pass A on a staged tile (see issue_tile for the layout)
template <class T>
__device__ void pass_a_compute(const KParams<T>& kp, StepShared& sh, const SlotHdr<T>& H,
                               const unsigned char* stage, const PipeLayout& L) {
  const Blk<T>& b = H.b;
  const Blk<T>& P = H.P;
  const Tile td = H.td;
  const int p = H.p, q = p ^ 1, sn = H.sn, SW = L.SW;
  const T* sE = reinterpret_cast<const T*>(stage);
  const T* sM = sE + (size_t)SW * kp.ty;
  const T* sN = sM + (size_t)SW * kp.ty;
  const T* sH = sN + (size_t)SW * (kp.ty + 1);
  const T* sX = sH + (size_t)SW * kp.ty;
  const bool child = b.is_child;
  T vol_t = T(0);  // this thread's cells; the tile reduction below is binary64
  double clip = 0.0, out = 0.0, ring = 0.0;
  bool bad = false;
  const int xe = min(td.x0 + kp.tx, b.nx), ye = min(td.y0 + kp.ty, b.ny);
  for (int j = td.y0 + threadIdx.y; j < ye; j += 8) {
    for (int i = td.x0 + threadIdx.x; i < xe; i += 32) {
      const int k = (j - td.y0) * SW + (i - td.x0);
      const T Mw = (child && i == 0) ? face_m(b, P, p, 0, j) : sM[k];
      const T Me = (child && i == b.nx - 1) ? face_m(b, P, p, b.nx, j) : sM[k + 1];
      const T Ns = (child && j == 0) ? face_n(b, P, p, i, 0) : sN[k];
      const T Nn = (child && j == b.ny - 1) ? face_n(b, P, p, i, b.ny) : sN[k + SW];
      if (child) {  // store the pulled edge fluxes for pass B
        if (i == 0) b.M[p][ix(b, 0, j)] = Mw;
        if (i == b.nx - 1) b.M[p][ix(b, b.nx, j)] = Me;
        if (j == 0) b.N[p][ix(b, i, 0)] = Ns;
        if (j == b.ny - 1) b.N[p][ix(b, i, b.ny)] = Nn;
      }
      const T h = sH[k];
      T e = sE[k] - (b.dtdx * (Me - Mw) + b.dtdx * (Nn - Ns));
      if (h + e < T(0)) {
        clip += (double)(-h - e) * b.dx2;
        e = -h;
      }
      if (td.flags & kTfRing) {
        T rv;
        if (ring_value(kp, b, p, i, j, h, rv)) {
          ring += ((double)rv - (double)e) * b.dx2;
          e = rv;
        }
      }
      const size_t c = ix(b, i, j);
      b.eta[q][c] = e;
      const T em = sX[k];
      if (h + e > b.eps && e > em) {
        if (em < b.thr && e >= b.thr) b.arr[c] = sn;
        b.emax[c] = e;
      }
      vol_t += e;
      if (i == 0) out += b.vol * (double)(-Mw);
      if (i == b.nx - 1) out += b.vol * (double)Me;
      if (j == 0) out += b.vol * (double)(-Ns);
      if (j == b.ny - 1) out += b.vol * (double)Nn;
      bad |= !dfinite(e);
    }
  }
  if (bad) atomicOr(b.status, kStNonFinite);
  const double vol = warp_sum((double)vol_t);
  clip = warp_sum(clip);
  out = warp_sum(out);
  ring = warp_sum(ring);
  const int w = threadIdx.y;
  if (threadIdx.x == 0) {
    sh.red[0][w] = vol;
    sh.red[1][w] = clip;
    sh.red[2][w] = out;
    sh.red[3][w] = ring;
  }
  __syncthreads();
  if (threadIdx.y == 0 && threadIdx.x < 4) {
    double a = 0.0;
    for (int k = 0; k < 8; ++k) a += sh.red[threadIdx.x][k];
    double* slot = b.budget + 4 * (size_t)((td.y0 / kp.ty) * b.tiles_x + td.x0 / kp.tx);
    if (threadIdx.x == 0) slot[0] = a;
    else slot[threadIdx.x] += a;
  }
}

// pass B on a staged tile: face terms into the derived arrays, then the face updates
template <class T>
__device__ void pass_b_compute(const KParams<T>& kp, const SlotHdr<T>& H, unsigned char* stage,
                               unsigned char* derived, const PipeLayout& L) {
  const Blk<T>& b = H.b;
  const Tile td = H.td;
  const int p = H.p, q = p ^ 1;
  const int W = L.SW;
  const size_t n = (size_t)L.SW * L.SH;
  BTile<T> S;
  S.W = W;
  T* st = reinterpret_cast<T*>(stage);
  S.E = st;
  S.H = st + n;
  S.MX = st + 2 * n;
  S.NY = st + 3 * n;
  S.NM = reinterpret_cast<float*>(st + 4 * n);
  T* dv = reinterpret_cast<T*>(derived);
  S.QX = dv;
  S.RX = dv + n;
  S.SY = dv + 2 * n;
  S.TY = dv + 3 * n;
  S.VX = reinterpret_cast<unsigned char*>(dv + 4 * n);
  S.VY = S.VX + n;
  const int ox = td.x0 - 4, oy = td.y0 - 2;  // global (c, r) of local (0, 0)
  // face terms of columns x0-1..x0+tx and rows y0-1..y0+ty
  for (int ly = 1 + threadIdx.y; ly <= kp.ty + 2; ly += 8) {
    for (int lx = 3 + threadIdx.x; lx <= kp.tx + 4; lx += 32) {
      const int k = ly * W + lx;
      const int c = ox + lx, r = oy + ly;
      {  // x-face (c, r)
        const T dep = T(0.5) * (S.H[k - 1] + S.H[k]) + T(0.5) * (S.E[k - 1] + S.E[k]);
        const bool interior = c >= 1 && c <= b.nx - 1 && r >= 0 && r <= b.ny - 1;
        S.VX[k] = interior && dep > b.eps;
        if (interior && dep != T(0)) {
          const T mm = S.MX[k];
          const T nb = T(0.25) * ((S.NY[k - 1] + S.NY[k]) + (S.NY[k - 1 + W] + S.NY[k + W]));
          S.QX[k] = Ar<T>::quot(mm * mm, dep);
          S.RX[k] = Ar<T>::quot(mm * nb, dep);
        }
      }
      {  // y-face (c, r)
        const T dep = T(0.5) * (S.H[k - W] + S.H[k]) + T(0.5) * (S.E[k - W] + S.E[k]);
        const bool interior = r >= 1 && r <= b.ny - 1 && c >= 0 && c <= b.nx - 1;
        S.VY[k] = interior && dep > b.eps;
        if (interior && dep != T(0)) {
          const T v = S.NY[k];
          const T mb = T(0.25) * ((S.MX[k - W] + S.MX[k]) + (S.MX[k - W + 1] + S.MX[k + 1]));
          S.SY[k] = Ar<T>::quot(v * v, dep);
          S.TY[k] = Ar<T>::quot(v * mb, dep);
        }
      }
    }
  }
  __syncthreads();
  T* Mo = b.M[q];
  T* No = b.N[q];
  const bool root = !b.is_child;
  const int xe = min(td.x0 + kp.tx, b.nx), ye = min(td.y0 + kp.ty, b.ny);
  for (int j = td.y0 + threadIdx.y; j < ye; j += 8) {
    for (int i = td.x0 + threadIdx.x; i < xe; i += 32) {
      const int k = (j - oy) * W + (i - ox);
      if (i >= 1) {
        Mo[ix(b, i, j)] = xmom_s(b, S, k);
      } else if (root) {
        Mo[ix(b, 0, j)] = b.bc[0] == kBcRadiation ? radiate_s(b, S, k, T(-1)) : T(0);
      }
      if (i == b.nx - 1 && root)
        Mo[ix(b, b.nx, j)] = b.bc[1] == kBcRadiation ? radiate_s(b, S, k, T(1)) : T(0);
      if (j >= 1) {
        No[ix(b, i, j)] = ymom_s(b, S, k);
      } else if (root) {
        No[ix(b, i, 0)] = b.bc[2] == kBcRadiation ? radiate_s(b, S, k, T(-1)) : T(0);
      }
      if (j == b.ny - 1 && root)
        No[ix(b, i, b.ny)] = b.bc[3] == kBcRadiation ? radiate_s(b, S, k, T(1)) : T(0);
    }
  }
}

// One pass over this CTA's tiles (t = blockIdx.x + k * gridDim.x) with two stages.
// Returns false when a wait ran out (kStTimeout recorded, copies drained).
template <class T>
__device__ bool run_pass(const KParams<T>& kp, StepShared& sh, unsigned char* dsm,
                         const PipeLayout& L, unsigned& phase, int s, bool passB) {
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(dsm);
  SlotHdr<T>* hdr = reinterpret_cast<SlotHdr<T>*>(dsm + 2 * sizeof(unsigned long long));
  unsigned char* stg[2] = {dsm + L.hdr, dsm + L.hdr + L.stage};
  unsigned char* derived = dsm + L.hdr + 2 * L.stage;
  IssueCache<T>& cache = *reinterpret_cast<IssueCache<T>*>(
      dsm + 2 * sizeof(unsigned long long) + 2 * sizeof(SlotHdr<T>));
  const int nt = *kp.ntiles;
  const int G = gridDim.x;
  const bool issuer = threadIdx.y == 0;
  int t = blockIdx.x;
  if (issuer && t < nt) {
    fence_proxy_async();  // earlier generic writes (other CTAs, previous pass) before the copies
    issue_tile(kp, t, s, passB, hdr[0], cache, stg[0], &bar[0], L);
  }
  for (int k = 0; t < nt; ++k, t += G) {
    const int st = k & 1;
    if (issuer && t + G < nt) {
      fence_proxy_async();  // this CTA's reads of the other stage before its refill
      issue_tile(kp, t + G, s, passB, hdr[st ^ 1], cache, stg[st ^ 1], &bar[st ^ 1], L);
    }
    const unsigned par = (phase >> st) & 1u;
    bool ok = mbar_wait(&bar[st], par, kp.spin_cycles);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0 && threadIdx.y == 0) atomicOr(kp.status, kStTimeout);
      mbar_wait(&bar[st], par, kp.spin_cycles);  // drain before leaving
      if (issuer && t + G < nt) mbar_wait(&bar[st ^ 1], (phase >> (st ^ 1)) & 1u, kp.spin_cycles);
      return false;
    }
    phase ^= 1u << st;
    if (hdr[st].active) {
      if (passB) pass_b_compute(kp, hdr[st], stg[st], derived, L);
      else pass_a_compute(kp, sh, hdr[st], stg[st], L);
    }
    __syncthreads();  // stage st and its header are free again
  }
  return true;
}

template <class T>
__device__ __forceinline__ void init_pipe(unsigned char* dsm) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(dsm);
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    reinterpret_cast<IssueCache<T>*>(dsm + 2 * sizeof(unsigned long long) +
                                     2 * sizeof(SlotHdr<T>))->blk = -1;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ device-wide barrier
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Sense-by-generation barrier over all CTAs of a cooperative launch. The wait is
// bounded: after spin_cycles the CTA records kStTimeout and every CTA leaves.
__device__ __forceinline__ bool grid_barrier(Bar* bar, unsigned& gen, int* status,
                                             long long spin_cycles, int* go) {
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const unsigned g = gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u) + 1u;
    bool ok = true;
    if (arrived == gridDim.x) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_u32(&bar->gen) == g) {
        if (clock64() - t0 > spin_cycles) {
          atomicOr(status, kStTimeout);
          ok = false;
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
    gen = g + 1;
    *go = ok && !(*(volatile int*)status & kStTimeout);
  }
  __syncthreads();
  return *go != 0;
}

// ------------------------------------------------------------------ kernels
// Dynamic shared memory of the step kernels: pipe_layout<T>(tx, ty).total bytes.
template <class T>
__global__ void __launch_bounds__(256) k_persistent(KParams<T> kp) {
  __shared__ StepShared sh;
  extern __shared__ __align__(128) unsigned char dsm[];
  const PipeLayout L = pipe_layout<T>(kp.tx, kp.ty);
  init_pipe<T>(dsm);
  unsigned phase = 0;
  unsigned gen = 0;
  if (threadIdx.x == 0 && threadIdx.y == 0) gen = ld_acquire_u32(&kp.bar->gen);
  for (int s = 0; s < kp.nsteps; ++s) {
    if (!run_pass(kp, sh, dsm, L, phase, s, false)) return;
    if (!grid_barrier(kp.bar, gen, kp.status, kp.spin_cycles, &sh.go)) return;
    if (!run_pass(kp, sh, dsm, L, phase, s, true)) return;
    if (s + 1 < kp.nsteps && !grid_barrier(kp.bar, gen, kp.status, kp.spin_cycles, &sh.go))
      return;
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_pass_a(KParams<T> kp, int s) {
  __shared__ StepShared sh;
  extern __shared__ __align__(128) unsigned char dsm[];
  const PipeLayout L = pipe_layout<T>(kp.tx, kp.ty);
  init_pipe<T>(dsm);
  unsigned phase = 0;
  run_pass(kp, sh, dsm, L, phase, s, false);
}

template <class T>
__global__ void __launch_bounds__(256) k_pass_b(KParams<T> kp, int s) {
  __shared__ StepShared sh;
  extern __shared__ __align__(128) unsigned char dsm[];
  const PipeLayout L = pipe_layout<T>(kp.tx, kp.ty);
  init_pipe<T>(dsm);
  unsigned phase = 0;
  run_pass(kp, sh, dsm, L, phase, s, true);
}

// sum(eta) of every tile at the current level (after an initial condition or a restore)
template <class T>
__global__ void __launch_bounds__(256) k_snapshot(KParams<T> kp) {
  __shared__ Blk<T> sb;
  __shared__ double red[8];
  const int nt = *kp.ntiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const Tile td = kp.tiles[t];
    __syncthreads();
    stage_blk(&sb, &RTI_BLK(kp, td.blk));
    __syncthreads();
    const int p = (int)(kp.scen[sb.scen].base & 1);
    double vol = 0.0;
    const int xe = min(td.x0 + kp.tx, sb.nx), ye = min(td.y0 + kp.ty, sb.ny);
    for (int j = td.y0 + threadIdx.y; j < ye; j += 8)
      for (int i = td.x0 + threadIdx.x; i < xe; i += 32) vol += (double)sb.eta[p][ix(sb, i, j)];
    vol = warp_sum(vol);
    if (threadIdx.x == 0) red[threadIdx.y] = vol;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      double a = 0.0;
      for (int k = 0; k < 8; ++k) a += red[k];
      sb.budget[4 * (size_t)((td.y0 / kp.ty) * sb.tiles_x + td.x0 / kp.tx)] = a;
    }
  }
}

// Store the coarse-to-fine edge fluxes of every child block into its current flux
// arrays (parity p), exactly as pass A of the next step will pull them. Used before a
// checkpoint read so that the child's edge faces hold their defined values.
template <class T>
__global__ void __launch_bounds__(256) k_fill_edges(KParams<T> kp, int p) {
  __shared__ Blk<T> sb, sP;
  const int nt = *kp.ntiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const Tile td = kp.tiles[t];
    __syncthreads();
    stage_blk(&sb, &RTI_BLK(kp, td.blk));
    __syncthreads();
    if (!sb.is_child) continue;
    stage_blk(&sP, &RTI_BLK(kp, sb.parent));
    __syncthreads();
    const int xe = min(td.x0 + kp.tx, sb.nx), ye = min(td.y0 + kp.ty, sb.ny);
    for (int j = td.y0 + threadIdx.y; j < ye; j += 8) {
      for (int i = td.x0 + threadIdx.x; i < xe; i += 32) {
        if (i == 0) sb.M[p][ix(sb, 0, j)] = face_m(sb, sP, p, 0, j);
        if (i == sb.nx - 1) sb.M[p][ix(sb, sb.nx, j)] = face_m(sb, sP, p, sb.nx, j);
        if (j == 0) sb.N[p][ix(sb, i, 0)] = face_n(sb, sP, p, i, 0);
        if (j == sb.ny - 1) sb.N[p][ix(sb, i, sb.ny)] = face_n(sb, sP, p, i, sb.ny);
      }
    }
  }
}

// end of a chunk: every scenario advances by the steps it took
__global__ void k_advance(ScenDev* sc, const int* nscen, int nsteps);

}  // namespace rti
