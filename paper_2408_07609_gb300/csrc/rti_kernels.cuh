// rti_kernels.cuh -- sm_103a kernels of the nested TUNAMI-N2 leap-frog step.
//
// Included by rti_fp32.cu and rti_fp64.cu, which instantiate it for binary32 and
// binary64 state. One time step is one sweep over a work list of strips (28 columns x
// ty rows of one block) that covers every block of every scenario in a batch. A warp
// steps a strip by marching up its rows and, at each row, computes
//
//   the mass update (Eq. 1, Sec. IV-A "NLMASS"): eta^{n+1} = eta^n - dt/dx (dM + dN),
//     the dry clip, the coarse-to-fine edge fluxes of a child (pulled from the
//     parent's current fluxes), the fine-to-coarse ring of a parent (Listing 5 mean of
//     the 3x3 child cells, recomputed from the child's stable time level), max height
//     and arrival (output update) and the binary64 volume budget (warp-shuffle sums);
//   the momentum update of the row below (Eqs. 2-3, "NLMNT2"/XMMT/YMMT): M^{n+1},
//     N^{n+1} with upwind advection, pressure on the total depth, semi-implicit
//     Manning friction, the wet/dry front and the outflow limit; radiation or wall
//     faces on root edges.
//
// eta, M and N are ping-ponged (parity = step & 1): a step reads level p and writes
// level p ^ 1, and every pull reads a level that no strip of the step modifies.
// The discrete rules follow the oracle's readings R1-R10 operation for operation;
// the binary64 build uses -fmad=false so that it rounds like the oracle.
//
// Block descriptors: a warp copies its strip's block descriptor (and, for a child, its
// parent's) into shared memory and reads fields from there. Optimised binary64 builds
// of an earlier kernel that re-read descriptor fields through references into the
// device table faulted on an in-range edge read (the range-checked, -G and
// copied-descriptor builds did not); the mixed-sequence GPU test guards this.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#include "rti_layout.h"

namespace rti {

__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }

// Cube root of the friction term's D^(7/3) in binary64: Newton-Raphson iteration for the
// reciprocal cube root (no division), the stated method the FP64 oracle uses too, so that
// with -fmad=false every operation rounds identically on both sides. x = m 2^e with m in
// [0.5, 1) and e = 3q + r (r in {0, 1, 2}); a = m 2^r; a quadratic least-squares start
// for m^(-1/3) scaled by 2^(-r/3); three steps y <- y + y (1 - a y^3) / 3; the result
// (a y) y times the exact power 2^q. For a positive normal x (other inputs only reach
// values the caller discards).
__device__ __forceinline__ double cube_root_nr(double x) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ffull) - 1022;
  const double m =
      __longlong_as_double((long long)((bits & 0x800fffffffffffffull) | (1022ull << 52)));
  const int q = e >= 0 ? e / 3 : -((2 - e) / 3);
  const int r = e - 3 * q;
  const double a = r == 0 ? m : (r == 1 ? m * 2.0 : m * 4.0);
  const double sc = r == 0 ? 1.0 : (r == 1 ? 0.7937005259840998 : 0.6299605249474366);
  double y = (1.7375834500937248 + m * (-1.1916185163999664 + m * 0.4564206970782672)) * sc;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t = y * y;
    t = t * y;
    t = a * t;
    t = 1.0 - t;
    t = y * t;
    t = t * 0.3333333333333333;
    y = y + t;
  }
  double c = a * y;
  c = c * y;
  const int qe = (q + 1023) & 0x7ff;  // (an out-of-range q only comes with a discarded x)
  return c * __longlong_as_double((long long)((unsigned long long)qe << 52));
}
// finite <=> the exponent field is not all ones (integer test, no conversions)
__device__ __forceinline__ bool dfinite(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ULL) !=
         0x7ff0000000000000ULL;
}
__device__ __forceinline__ bool dfinite(float x) {
  return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
}

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
// (2 v_k + v_n) / 3 in the state precision: binary64 as the oracle writes it, binary32
// in binary32 (a binary64 divide costs dozens of slow FP64 instructions on this part).
__device__ __forceinline__ double interp3(double vk, double vn) { return (2.0 * vk + vn) / 3.0; }
__device__ __forceinline__ float interp3(float vk, float vn) { return (2.0f * vk + vn) / 3.0f; }

// Fine face t of an edge whose coarse faces are v(k), k = 0..K-1: the coarse value at
// the middle fine face, (2 v_k + v_{k+-1}) / 3 at the outer ones, neighbour clamped;
// with `constant` every fine face takes v_k.
template <class T>
__device__ __forceinline__ T edge_interp(const T* arr, const Blk<T>& P, int fixed, int start,
                                         int K, int t, bool along_y, bool constant) {
  int k = t / 3, sub = t - 3 * k;
  const T vk = along_y ? arr[ix(P, fixed, start + k)] : arr[ix(P, start + k, fixed)];
  if (sub == 1 || constant) return vk;
  int kn = sub == 0 ? k - 1 : k + 1;
  kn = kn < 0 ? 0 : (kn > K - 1 ? K - 1 : kn);
  const T vn = along_y ? arr[ix(P, fixed, start + kn)] : arr[ix(P, start + kn, fixed)];
  return interp3(vk, vn);
}

// x-flux of face (f, j) at parity p; a child's edge faces come from its parent P.
template <class T>
__device__ __forceinline__ T face_m(const Blk<T>& b, const Blk<T>& P, int p, int f, int j) {
  if (b.is_child && (f == 0 || f == b.nx)) {
    int F = b.i0 + (f == 0 ? 0 : b.nx / 3);
    return edge_interp<T>(P.M[p], P, F, b.j0, b.ny / 3, j, true, (b.nest & kNestConst) != 0);
  }
  return b.M[p][ix(b, f, j)];
}
template <class T>
__device__ __forceinline__ T face_n(const Blk<T>& b, const Blk<T>& P, int p, int i, int g) {
  if (b.is_child && (g == 0 || g == b.ny)) {
    int G = b.j0 + (g == 0 ? 0 : b.ny / 3);
    return edge_interp<T>(P.N[p], P, G, b.i0, b.nx / 3, i, false, (b.nest & kNestConst) != 0);
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
// Patch (u, v) of child c (parent cell (c.i0 + u, c.j0 + v) of block P, on the inner
// ring of c's footprint, or anywhere on it with full feedback): if the 3x3 child patch
// has a wet cell, `out` gets the mean of
// the wet child levels at eta^{n+1} (recomputed from the child's level p; binary64
// accumulator, Listing 5 order: x outer, y inner), floored at -hP.
template <class T>
__device__ bool ring_patch(const Blk<T>& c, const Blk<T>& P, int p, int u, int v, T hP, T& out) {
  constexpr double kInvWet[10] = {0.0,       1.0 / 1.0, 1.0 / 2.0, 1.0 / 3.0, 1.0 / 4.0,
                                  1.0 / 5.0, 1.0 / 6.0, 1.0 / 7.0, 1.0 / 8.0, 1.0 / 9.0};
  double sum = 0.0;
  int wet = 0;
  for (int x = 3 * u; x < 3 * u + 3; ++x) {    // outer: x (the paper's J)
    for (int y = 3 * v; y < 3 * v + 3; ++y) {  // inner: y (the paper's I)
      T e = child_eta_next(c, P, p, x, y);
      if (c.h[ix(c, x, y)] + e > c.eps) {
        sum = sum + (double)e;
        wet = wet + 1;
      }
    }
  }
  if (wet == 0) return false;
  double avg = sum * kInvWet[wet];  // = sum * (1.0 / wet): the table holds the rounded quotients
  if (avg < -(double)hP) avg = -(double)hP;
  out = (T)avg;
  return true;
}

// "no override" in a ring plane: all-ones bits (a NaN that arithmetic never produces
// from finite data and that the kernels test by its bits)
__device__ __forceinline__ bool ring_unset(float v) { return __float_as_uint(v) == 0xffffffffu; }
__device__ __forceinline__ bool ring_unset(double v) {
  return __double_as_longlong(v) == (long long)-1;
}
__device__ __forceinline__ float ring_none(float) { return __uint_as_float(0xffffffffu); }
__device__ __forceinline__ double ring_none(double) { return __longlong_as_double(-1LL); }

// ------------------------------------------------------------------ momentum (R2-R4, R6)
// First-order upwind difference on the sign of w (w = 0: the centred difference);
// a difference that needs an unusable face is 0. Written as selects so that the
// compiler can interleave the x and y updates.
template <class T>
__device__ __forceinline__ T upwind(T w, T phim, T phi0, T phip, bool okm, bool okp) {
  const T pos = okm ? phi0 - phim : T(0);
  const T neg = okp ? phip - phi0 : T(0);
  const T mid = (okm && okp) ? T(0.5) * (phip - phim) : T(0);
  return w > T(0) ? pos : (w < T(0) ? neg : mid);
}

// Arithmetic of the momentum update in the state precision. Binary64 keeps the oracle's
// exact expressions (correctly rounded divide and square root, the stated cube-root
// iteration cube_root_nr) so that it reproduces the oracle's rounding bit for bit.
// Binary32 (the forecast path, checked against the oracle within the stated accuracy)
// uses the special-function unit: approximate reciprocals, and sqrt(M^2 + N^2) D^(-7/3)
// = 2^(log2(M^2 + N^2)/2 - 7/3 log2 D) with the PTX lg2.approx / ex2.approx instructions
// (log2 0 = -inf gives a zero friction).
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Constants of the momentum update of one block, formed once per strip: binary64 keeps
// the oracle's factors, binary32 folds the loop-invariant products and quotient.
template <class T>
struct MomK;
template <>
struct MomK<double> {
  double eps, dtdx, g, cfric, dx, q4dt, vlim;
};
template <>
struct MomK<float> {
  float eps, dtdx, gdtdx /* g dt/dx */, cfric, dxq /* dx / (4 dt) */, vlim;
};
template <class T>
__device__ __forceinline__ MomK<T> mom_consts(const Blk<T>& b);
template <>
__device__ __forceinline__ MomK<double> mom_consts(const Blk<double>& b) {
  return MomK<double>{b.eps, b.dtdx, b.g, b.cfric, b.dx, b.q4dt, b.vlim};
}
template <>
__device__ __forceinline__ MomK<float> mom_consts(const Blk<float>& b) {
  return MomK<float>{b.eps, b.dtdx, b.g * b.dtdx, b.cfric, b.dx / b.q4dt, b.vlim};
}

template <class T>
struct Ar;
template <>
struct Ar<double> {
  static constexpr bool kSelect = false;  // divide only where the quotient is used
  static __device__ __forceinline__ void quot2(double a1, double a2, double b, double& q1,
                                               double& q2) {
    q1 = a1 / b;
    q2 = a2 / b;
  }
  static __device__ __forceinline__ double update(double m, double across, double Df,
                                                  double grad, double adv, double nf,
                                                  const MomK<double>& K) {
    double P = K.g * Df * K.dtdx * grad;
    double F = K.cfric * nf * nf * sqrt(m * m + across * across) / (Df * Df * cube_root_nr(Df));
    return ((1.0 - F) * m - adv - P) / (1.0 + F);
  }
  // R11: velocity across a face of flux q and depth D (0 on a face without water)
  static __device__ __forceinline__ double face_vel(double q, double D, double eps) {
    return D > eps ? q / D : 0.0;
  }
  // Outflow limit: |flux| <= D dx / (4 dt) with D the depth of the cell it drains, and
  // with the velocity limit (kernel variant kLim) also |flux| <= vlim Df.
  template <bool kLim>
  static __device__ __forceinline__ double limit(double m, double Dlo, double Dhi, double Df,
                                                 const MomK<double>& K) {
    double cap = (m > 0.0 ? Dlo : Dhi) * K.dx / K.q4dt;
    if (kLim) {
      const double vc = K.vlim * Df;
      if (vc < cap) cap = vc;
    }
    if (m > cap) return cap;
    if (m < -cap) return -cap;
    return m;
  }
};
template <>
struct Ar<float> {
  static constexpr bool kSelect = true;  // divide everywhere and select (no branch)
  static __device__ __forceinline__ void quot2(float a1, float a2, float b, float& q1,
                                               float& q2) {
    const float r = __fdividef(1.0f, b);
    q1 = a1 * r;
    q2 = a2 * r;
  }
  static __device__ __forceinline__ float update(float m, float across, float Df, float grad,
                                                 float adv, float nf, const MomK<float>& K) {
    const float P = K.gdtdx * Df * grad;
    const float s2 = m * m + across * across;
    const float F =
        (K.cfric * nf * nf) * ex2_approx(0.5f * lg2_approx(s2) - 2.33333333f * lg2_approx(Df));
    return __fdividef((1.0f - F) * m - adv - P, 1.0f + F);
  }
  static __device__ __forceinline__ float face_vel(float q, float D, float eps) {
    return D > eps ? __fdividef(q, D) : 0.0f;
  }
  template <bool kLim>
  static __device__ __forceinline__ float limit(float m, float Dlo, float Dhi, float Df,
                                                const MomK<float>& K) {
    float cap = (m > 0.0f ? Dlo : Dhi) * K.dxq;
    if (kLim) cap = fminf(cap, K.vlim * Df);
    if (m > cap) return cap;  // (a NaN passes through, for the non-finite check)
    if (m < -cap) return -cap;
    return m;
  }
};

// ------------------------------------------------------------------ block reduction
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ the fused step
// A step is one sweep over strips. A strip is kStripW columns x ty rows of one block
// and is stepped by one warp: lane L holds column c = x0 - 2 + L; lanes 2..29 own the
// strip's cells and faces, lanes 0, 1, 30 and 31 recompute the halo that the stencils
// read. The warp marches up the rows. At row r it loads eta^n, h, M^n, N^n (of the face
// above), eta_max and Manning n; forms eta^{n+1} of row r (Eq. 1 with the dry clip,
// the pulled child-edge fluxes and the ring mean), stores it with the output update of
// the owned cells, and forms the advective face terms of row r. It then updates the
// fluxes of row r - 1 (Eqs. 2-3), whose stencil -- eta^{n+1} and face terms of rows
// r-2..r, columns c-1..c+1 -- is complete in its registers and its neighbours'.
// The two passes of the paper's step (mass, then momentum) thus become one sweep in
// which eta^{n+1} is recomputed on the halo instead of being stored and re-read; the
// arithmetic of every value is the same expression in the same order.

// One row of a lane's column as the march carries it (record of row r, cell (c, r),
// x-face (c, r) between cells c-1 and c, y-face (c, r) between rows r-1 and r).
template <class T>
struct Row {
  T E, H;        // eta^{n+1}, h of cell (c, r)
  T eL, hL;      // the same of cell (c - 1, r)
  T MX, mE;      // M^n of x-faces (c, r) and (c + 1, r)
  T NY;          // N^n of y-face (c, r)
  T nb;          // N-bar of x-face (c, r)
  T QX, RX;      // M^2/D and M N-bar/D of x-face (c, r)
  T mb;          // M-bar of y-face (c, r)
  T SY, TY;      // N^2/D and N M-bar/D of y-face (c, r)
  float nm;      // Manning n of cell (c, r)
  unsigned fl;   // bit 0: x-face (c, r), bit 1: y-face (c, r) is interior with D > dry_eps
                 // (usable by advection)
};

// Raw inputs of row r: eta^n, h, M^n, eta_max, Manning n of (c, r); N^n of y-face (c, r+1).
template <class T>
struct Raw {
  T e, h, m, nn, em;
  float nm;
  T vm;      // squared-speed maximum (velocity tracking only)
  T eN, hN;  // eta^n and h of cell (c, r + 1) (velocity tracking only)
  T rv;      // ring-plane entry of cell (c, r) (ring strips only)
};

// The march's input rows are staged ahead in shared memory: a ring of kRingD slots per
// warp, each holding elements [x0 - 4, x0 + 32) of the six input rows of one row r.
// 16-byte cp.async.cg copies (through L2, no registers held) keep kRingD - 2 rows per
// warp in flight; a slot is refilled two rows after it was read, so one __syncwarp per
// row orders the reads before the refill. A copy that would start past the allocated
// row is a zero fill.
// slots per warp, a power of two (slots are taken modulo by a mask): binary64 is bound by
// its arithmetic and keeps fewer rows in flight, inside the 48 KB of static shared memory
template <class T>
struct RingD {
  static constexpr int D = 8;
};
template <>
struct RingD<double> {
  static constexpr int D = 4;
};
constexpr int kRingW = 36;

template <class T, bool kRg>
struct __align__(16) RingSlot {
  T e[kRingW], h[kRingW], m[kRingW], nn[kRingW], em[kRingW];
  float nm[kRingW];
  T vm[kRingW];  // squared-speed maximum, staged only when the block tracks it
  T rg[kRingW];  // ring-plane entries (ring strips of full-feedback variants)
};
template <class T>
struct __align__(16) RingSlot<T, false> {  // the other variants read the ring plane directly
  T e[kRingW], h[kRingW], m[kRingW], nn[kRingW], em[kRingW];
  float nm[kRingW];
  T vm[kRingW];
};

// One 16-byte copy, issued only where `issue` holds (a predicate on the instruction, not
// a branch); `valid` false makes it a zero fill that reads nothing.
__device__ __forceinline__ void cp_async16(bool issue, void* sdst, const void* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  const int n = valid ? 16 : 0;
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %3, 0;\n\t"
      "@p cp.async.cg.shared.global [%0], [%1], 16, %2;\n\t}" ::"r"(d),
      "l"(gsrc), "r"(n), "r"((int)issue)
      : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Lanes issue the 16-byte chunks of row r (element `rowbase` = (r + 2) pitch + x0 is the
// strip's column x0 - 4; N is taken one row up).
// What a lane copies of every staged row (fixed for a strip): chunk k of the state
// arrays and of Manning n, whether it has one, and whether it lies inside the row.
struct StageLane {
  int ke, km;
  bool ie, oe, im, om;
};
template <class T>
__device__ __forceinline__ StageLane stage_lane(int lane, int x0, int pitch) {
  constexpr int E = 16 / (int)sizeof(T);  // elements per chunk
  constexpr int NC = kRingW / E;          // chunks per row of a state array
  constexpr int NM = kRingW / 4;          // chunks of Manning n (binary32)
  static_assert(NC <= 32, "one chunk per lane");
  StageLane L;
  L.ie = lane < NC;
  L.ke = (L.ie ? lane : NC - 1) * E;
  L.oe = x0 + L.ke + E <= pitch;
  L.im = lane < NM;
  L.km = (L.im ? lane : NM - 1) * 4;
  L.om = x0 + L.km + 4 <= pitch;
  return L;
}

// The five state-array chunks of a lane under one predicate: shared destinations kRingW
// elements (STRIDE bytes) apart from `d`.
template <int STRIDE>
__device__ __forceinline__ void cp_async16x5(bool issue, unsigned d, const void* g0,
                                             const void* g1, const void* g2, const void* g3,
                                             const void* g4, bool valid) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
      "@p cp.async.cg.shared.global [%0], [%1], 16, %7;\n\t"
      "@p cp.async.cg.shared.global [%0+%8], [%2], 16, %7;\n\t"
      "@p cp.async.cg.shared.global [%0+%9], [%3], 16, %7;\n\t"
      "@p cp.async.cg.shared.global [%0+%10], [%4], 16, %7;\n\t"
      "@p cp.async.cg.shared.global [%0+%11], [%5], 16, %7;\n\t}" ::"r"(d),
      "l"(g0), "l"(g1), "l"(g2), "l"(g3), "l"(g4), "r"((int)issue), "r"(valid ? 16 : 0),
      "n"(STRIDE), "n"(2 * STRIDE), "n"(3 * STRIDE), "n"(4 * STRIDE)
      : "memory");
}

template <class T, bool kTrack, bool kRg>
__device__ __forceinline__ void stage_row(RingSlot<T, kRg>& S, const T* eta, const T* h, const T* M,
                                          const T* N, const T* emax, const float* man,
                                          const T* vmax, const T* ring, int rowbase, int pitch,
                                          const StageLane& L, bool row_ok) {
  using Slot = RingSlot<T, kRg>;
  static_assert(offsetof(Slot, h) == kRingW * sizeof(T) &&
                    offsetof(Slot, em) == 4 * kRingW * sizeof(T),
                "state rows kRingW elements apart");
  const int g = L.oe ? rowbase + L.ke : rowbase;
  cp_async16x5<kRingW * (int)sizeof(T)>(row_ok && L.ie,
                                        (unsigned)__cvta_generic_to_shared(&S.e[L.ke]), eta + g,
                                        h + g, M + g, N + g + pitch, emax + g, L.oe);
  cp_async16(row_ok && L.im, &S.nm[L.km], man + (L.om ? rowbase + L.km : rowbase), L.om);
  if (kTrack) cp_async16(row_ok && L.ie, &S.vm[L.ke], vmax + g, L.oe);
  if constexpr (kRg) {
    if (ring) cp_async16(row_ok && L.ie, &S.rg[L.ke], ring + g, L.oe);
  }
}

template <class T, bool kTrack, bool kRg>
__device__ __forceinline__ Raw<T> read_row(const RingSlot<T, kRg>& S, int lane) {
  Raw<T> R;
  R.e = S.e[lane + 2];
  R.h = S.h[lane + 2];
  R.m = S.m[lane + 2];
  R.nn = S.nn[lane + 2];
  R.em = S.em[lane + 2];
  R.nm = S.nm[lane + 2];
  R.vm = kTrack ? S.vm[lane + 2] : T(0);
  return R;
}

// R2 + R4 at x-face (c, j): cells W = (c-1, j), E = (c, j); QX of faces c-1, c, c+1
// and RX of rows j-1, j, j+1 with their usable flags. Every case of the wet/dry rule is
// evaluated and the result selected (the values are those of the case analysis: a
// discarded case may produce a NaN that is never selected).
template <bool kLim, class T>
__device__ __forceinline__ T xmom_r(T hL, T eL, T hR, T eR, T m, T nb, bool okm, T qm, T q0,
                                    bool okp, T qp, bool oks, T rs, T r0, bool okn, T rn,
                                    float nL, float nR, const MomK<T>& K) {
  const T eps = K.eps, dtdx = K.dtdx;
  const bool wL = hL + eL > eps, wR = hR + eR > eps;
  const bool both = wL && wR;
  const bool oneL = wL && !wR && eL > -hR;  // water flows onto the dry east cell
  const bool oneR = wR && !wL && eR > -hL;  // water flows onto the dry west cell
  const T Df = both ? T(0.5) * (hL + hR) + T(0.5) * (eL + eR) : (oneL ? eL + hR : eR + hL);
  const T grad = both ? eR - eL : (oneL ? -hR - eL : eR + hL);
  const T ax = upwind(m, okm ? qm : T(0), q0, okp ? qp : T(0), okm, okp);
  const T ay = upwind(nb, oks ? rs : T(0), r0, okn ? rn : T(0), oks, okn);
  const T adv = both ? dtdx * (ax + ay) : T(0);
  const T nf = (T)(nL > nR ? nL : nR);
  const T m1 = Ar<T>::update(m, nb, Df, grad, adv, nf, K);
  const bool keep = (both || oneL || oneR) && Df > eps && (both || (wL ? !(m1 < T(0)) : !(m1 > T(0))));
  const T lim = Ar<T>::template limit<kLim>(m1, hL + eL, hR + eR, Df, K);
  return keep ? lim : T(0);
}

// R3 + R4 at y-face (c, j): cells S = (c, j-1), N = (c, j); SY of rows j-1, j, j+1 and
// TY of faces c-1, c, c+1 with their usable flags (selects as in xmom_r).
template <bool kLim, class T>
__device__ __forceinline__ T ymom_r(T hS, T eS, T hN, T eN, T v, T mb, bool okm, T sm, T s0,
                                    bool okp, T sp, bool okw, T tw, T t0, bool oke, T te,
                                    float nS, float nN, const MomK<T>& K) {
  const T eps = K.eps, dtdx = K.dtdx;
  const bool wS = hS + eS > eps, wN = hN + eN > eps;
  const bool both = wS && wN;
  const bool oneS = wS && !wN && eS > -hN;
  const bool oneN = wN && !wS && eN > -hS;
  const T Df = both ? T(0.5) * (hS + hN) + T(0.5) * (eS + eN) : (oneS ? eS + hN : eN + hS);
  const T grad = both ? eN - eS : (oneS ? -hN - eS : eN + hS);
  const T ay = upwind(v, okm ? sm : T(0), s0, okp ? sp : T(0), okm, okp);
  const T ax = upwind(mb, okw ? tw : T(0), t0, oke ? te : T(0), okw, oke);
  const T adv = both ? dtdx * (ay + ax) : T(0);
  const T nf = (T)(nS > nN ? nS : nN);
  const T v1 = Ar<T>::update(v, mb, Df, grad, adv, nf, K);
  const bool keep = (both || oneS || oneN) && Df > eps && (both || (wS ? !(v1 < T(0)) : !(v1 > T(0))));
  const T lim = Ar<T>::template limit<kLim>(v1, hS + eS, hN + eN, Df, K);
  return keep ? lim : T(0);
}

// Both cells wet and every face of both upwind stencils usable (the open-water case):
// the wet/dry cases and usable flags of xmom_r / ymom_r drop out. Same expressions, so
// the same values as the general form under those conditions.
template <class T>
__device__ __forceinline__ T upwind_open(T w, T phim, T phi0, T phip) {
  return w > T(0) ? phi0 - phim : (w < T(0) ? phip - phi0 : T(0.5) * (phip - phim));
}
template <bool kLim, class T>
__device__ __forceinline__ T mom_open(T hA, T eA, T hB, T eB, T m, T across, T pm, T p0, T pp,
                                      T qm, T q0, T qp, float nA, float nB, const MomK<T>& K) {
  const T Df = T(0.5) * (hA + hB) + T(0.5) * (eA + eB);
  const T grad = eB - eA;
  const T a1 = upwind_open(m, pm, p0, pp);
  const T a2 = upwind_open(across, qm, q0, qp);
  const T adv = K.dtdx * (a1 + a2);
  const T nf = (T)(nA > nB ? nA : nB);
  const T m1 = Ar<T>::update(m, across, Df, grad, adv, nf, K);
  // no Df > eps test: the open-water vote requires both faces of the update usable
  // (depth above dry_eps) on every lane whose result is stored
  return Ar<T>::template limit<kLim>(m1, hA + eA, hB + eB, Df, K);
}

// R6: flux leaving through a root edge next to a cell (sign +1 east/north, -1 west/south)
template <class T>
__device__ __forceinline__ T radiate_r(T h, T e, T sign, T eps, T g) {
  if (!(h + e > eps)) return T(0);
  return sign * (dsqrt(g * (h > T(0) ? h : T(0))) * e);
}

// Per-warp shared memory: the input ring, the strip's block descriptor (and its
// parent's), its scenario counters and the index of the block staged. The variants with
// full feedback (kFull) also stage the ring plane and keep the rows the patch means need;
// the others do without that shared memory (a larger footprint costs them L1 capacity).
template <class T, bool kFull>
struct WarpSlot {
  RingSlot<T, kFull> ring[RingD<T>::D];
  Blk<T> b;
  Blk<T> P;
  ScenDev sc;
  int blk;
  T fb[3][32];  // eta^{n+1} before the ring override, rows r mod 3 (kFull only)
};
template <class T>
struct WarpSlot<T, false> {
  RingSlot<T, false> ring[RingD<T>::D];
  Blk<T> b;
  Blk<T> P;
  ScenDev sc;
  int blk;
};

template <class T>
__device__ __forceinline__ void warp_copy(void* dst, const void* src, int bytes) {
  const unsigned* s = reinterpret_cast<const unsigned*>(src);
  unsigned* d = reinterpret_cast<unsigned*>(dst);
  for (int w = threadIdx.x; w < bytes / 4; w += 32) d[w] = s[w];
}

// Stage block `blk`'s descriptor (and its parent's) and scenario counters in the warp's
// slot, unless they are there already.
template <class T, class WS>
__device__ __forceinline__ void stage_strip(const KParams<T>& kp, WS& ws, int blk) {
  if (blk == ws.blk) return;
  __syncwarp();
  warp_copy<T>(&ws.b, &RTI_BLK(kp, blk), sizeof(Blk<T>));
  __syncwarp();
  if (ws.b.is_child) warp_copy<T>(&ws.P, &RTI_BLK(kp, ws.b.parent), sizeof(Blk<T>));
  if (threadIdx.x == 0) {
    ws.sc = kp.scen[ws.b.scen];
    ws.blk = blk;
  }
  __syncwarp();
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Bounded wait of one warp until the flags kp.done[list[0 .. n)] reach `target` (lanes
// poll some each, relaxed loads, sleeping between rounds up to 2 us; past spin_cycles the
// warp flags a timeout and gives up). Each lane's fence after its last poll, then the
// warp barrier, order the lanes' later loads after the flagged strips' stores.
template <class T>
__device__ __noinline__ void wait_flags(const KParams<T>& kp, const int* list, int n,
                                        unsigned long long target) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x;
  const long long t0 = clock64();
  unsigned ns = 64;
  bool gave_up = false;
  for (int k0 = 0; k0 < n && !gave_up; k0 += 32) {
    const int k = k0 + lane;
    const unsigned long long* f = k < n ? kp.done + list[k] : nullptr;
    bool ok = !f || ld_relaxed_u64(f) >= target;
    while (!__all_sync(full, ok)) {
      if (__shfl_sync(full, clock64() - t0 > kp.spin_cycles ? 1 : 0, 0)) {
        if (lane == 0) atomicOr(kp.status, kStTimeout);
        gave_up = true;
        break;
      }
      __nanosleep(ns);
      ns = ns < 2048 ? 2 * ns : ns;
      if (!ok) ok = ld_relaxed_u64(f) >= target;
    }
  }
  __threadfence();
  __syncwarp();
}

// Bounded wait of one warp until child c's patches [u0, u1) x [v0, v1) (parent cells
// relative to the footprint) hold their means of step s. Patch (u, v) belongs to the
// strip whose owned columns and rows hold its last cell (3u + 2, 3v + 2), which flags
// the step once it has ended. Each lane polls the flags of some of those strips with
// relaxed loads, sleeping between rounds (backing off up to 2 us, so
// that a waiting warp takes neither issue slots nor L2 bandwidth from the rest). Past
// `spin_cycles` (lane 0's clock decides for the warp) it flags a timeout in `status` and
// gives up: the state of the step is then undefined and the host reports the timeout.
// Each lane's fence after its last poll, then the warp barrier, order the lanes' later
// loads after the flagged strips' stores.
template <class T>
__device__ void wait_child_strips(const KParams<T>& kp, const Blk<T>& c, int u0, int u1,
                                  int v0, int v1, int s) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x;
  const int sx0 = (3 * u0 + 2) / kp.tx, sx1 = (3 * (u1 - 1) + 2) / kp.tx;  // inclusive
  const int sy0 = (3 * v0 + 2) / kp.ty, sy1 = (3 * (v1 - 1) + 2) / kp.ty;
  const int nxs = sx1 - sx0 + 1, n = nxs * (sy1 - sy0 + 1);
  const unsigned long long target = ((unsigned long long)s << 32) | kDoneAll;
  const long long t0 = clock64();
  unsigned ns = 128;
  bool gave_up = false;
  for (int k0 = 0; k0 < n && !gave_up; k0 += 32) {
    const int k = k0 + lane;
    const unsigned long long* f = kp.done + c.strip0 + (sy0 + k / nxs) * c.tiles_x + sx0 + k % nxs;
    bool ok = k >= n || ld_relaxed_u64(f) >= target;
    while (!__all_sync(full, ok)) {
      if (__shfl_sync(full, clock64() - t0 > kp.spin_cycles ? 1 : 0, 0)) {
        if (lane == 0) atomicOr(kp.status, kStTimeout);
        gave_up = true;
        break;
      }
      __nanosleep(ns);
      ns = ns < 2048 ? 2 * ns : ns;
      if (!ok) ok = ld_relaxed_u64(f) >= target;
    }
  }
  __threadfence();
  __syncwarp();
}

// A strip has ended step s of the chunk: the warp barrier orders its lanes' stores before
// lane 0's fence, which orders them before the flag.
__device__ __forceinline__ void strip_finished(unsigned long long* flag, int s) {
  __syncwarp();
  if (threadIdx.x == 0) {
    __threadfence();
    st_relaxed_u64(flag, ((unsigned long long)s << 32) | kDoneAll);
  }
}

// The ring strip `td` of a parent with full feedback waits until the means of its region
// (the rows and columns its march reads) are stored for step s: the child strips that
// own them come earlier in the work list, and they wait on nothing after them.
template <class T, class WS>
__device__ __noinline__ void wait_ring_means(const KParams<T>& kp, const WS& ws, Tile td, int s) {
  const Blk<T>& b = ws.b;
  const int ye = min(td.y0 + kp.ty, b.ny);
  const int c0 = max(td.x0 - 2, 0), c1 = min(td.x0 + kStripW + 2, b.nx);
  const int r0 = max(td.y0 - 2, 0), r1 = min(ye + 1, b.ny);
  for (int q = 0; q < b.child_count; ++q) {
    const Blk<T>& ch = RTI_BLK(kp, RTI_KID(kp, b.child_first + q));
    const int a0 = ch.i0, a1 = ch.i0 + ch.nx / 3, b0 = ch.j0, b1 = ch.j0 + ch.ny / 3;
    const int u0 = max(c0, a0) - a0, u1 = min(c1, a1) - a0;
    const int v0 = max(r0, b0) - b0, v1 = min(r1, b1) - b0;
    if (u0 < u1 && v0 < v1) wait_child_strips(kp, ch, u0, u1, v0, v1, s);
  }
}

// R8 with full feedback, formed by the child's own march (one patch of 3x3 child cells
// per parent cell). Strip rows r = 3v + 2 with y0 <= r < ye and owned lanes on columns
// c = 3u + 2 complete patch (u, v): its cells are rows r-2..r (the two records before
// row r and row r itself) and columns c-2..c (this lane and the two to its left), all of
// which the strip computes (lanes 0..29 hold correct levels, rows y0-2..ye). Each patch
// thus belongs to exactly one strip. In binary64 the sum runs in the oracle's order, x
// outer and y inner: the lane of the patch's first column adds its three wet levels to 0,
// the next lane continues from that sum, the third from the second's (a dry level adds
// +0.0, which leaves a sum that is never -0.0 unchanged), and the quotient is the
// correctly rounded 1/n: the oracle's bits. Binary32 sums each column and then the three
// column sums (the same terms, associated differently) and takes 1/n from a table of
// rounded quotients: fewer instructions, and none on the FP64 pipe. The mean over the wet
// cells, floored at -hP, or "none" goes to the parent's ring plane at (i0 + u, j0 + v).
// `a0`, `a1`, `a2` are the lane's levels of rows r-2, r-1, r before the block's own ring
// override, so that every level feeds back what it computed itself.
static __constant__ float kRecipCount[10] = {0.0f,        1.0f / 1.0f, 1.0f / 2.0f, 1.0f / 3.0f,
                                             1.0f / 4.0f, 1.0f / 5.0f, 1.0f / 6.0f, 1.0f / 7.0f,
                                             1.0f / 8.0f, 1.0f / 9.0f};

template <class T>
__device__ __forceinline__ void patch_means(const Blk<T>& b, const Blk<T>& P, T a0, T h0, T a1,
                                            T h1, T a2, T h2, bool last, int c, int r) {
  const unsigned full = 0xffffffffu;
  const bool w0 = h0 + a0 > b.eps, w1 = h1 + a1 > b.eps, w2 = h2 + a2 > b.eps;
  const T d0 = w0 ? a0 : T(0), d1 = w1 ? a1 : T(0), d2 = w2 ? a2 : T(0);
  T acc;
  if constexpr (sizeof(T) == 8) {
    acc = ((T(0) + d0) + d1) + d2;                          // the patch's first column
    acc = ((__shfl_up_sync(full, acc, 1) + d0) + d1) + d2;  // its second
    acc = ((__shfl_up_sync(full, acc, 1) + d0) + d1) + d2;  // its third: the sum
  } else {
    const T col = (d0 + d1) + d2;
    acc = (__shfl_up_sync(full, col, 2) + __shfl_up_sync(full, col, 1)) + col;
  }
  int n = (int)w0 + (int)w1 + (int)w2;
  n = n + __shfl_up_sync(full, n, 1) + __shfl_up_sync(full, n, 2);
  if (last) {
    const size_t o = ix(P, b.i0 + c / 3, b.j0 + r / 3);
    if (n == 0) {
      P.ring[o] = ring_none(T(0));
    } else {
      T avg;
      if constexpr (sizeof(T) == 8) avg = acc * (1.0 / (double)n);
      else avg = acc * kRecipCount[n];
      const T hP = P.h[o];
      if (avg < -hP) avg = -hP;
      P.ring[o] = avg;
    }
  }
}

// Prepass of a strip over the region its march reads: columns x0-2..x0+29, rows
// y0-2..ye of cells and x-faces, y-faces up to row ye+1. A child's edge faces there get
// the parent's current fluxes (R7), stored into the child's own level-p arrays, whose
// edge entries nothing else reads; a parent's ring cells there get their fine-to-coarse
// eta^{n+1} or "none" (R8) in the ring plane, recomputed from the child's level p on the
// inner ring of each child footprint (with full feedback the children's marches fill the
// plane for every covered cell: patch_means, wait_ring_means). The items of the region are spread over
// the lanes; strips that overlap store the same values, and __syncwarp orders the
// stores before the march's loads. Kept out of line so that the march's registers do
// not pay for the nesting arithmetic.
template <class T, class WS>
__device__ __noinline__ void strip_prepass(const KParams<T>& kp, const WS& ws, Tile td,
                                           int p) {
  const Blk<T>& b = ws.b;
  const int nx = b.nx, ny = b.ny;
  const int lane = threadIdx.x;
  const int ye = min(td.y0 + kp.ty, ny);
  const int cx0 = td.x0 - 2, cx1 = td.x0 + 30;  // columns [cx0, cx1)
  const int ry0 = td.y0 - 2, ry1 = ye + 1;      // cell rows [ry0, ry1); y-face rows [ry0, ry1]
  if (b.is_child) {
    const int r0 = max(ry0, 0), r1 = min(ry1, ny);
    for (int side = 0; side < 2; ++side) {  // west / east faces M(f, r)
      const int f = side ? nx : 0;
      if (f < cx0 || f >= cx1) continue;
      for (int r = r0 + lane; r < r1; r += 32) b.M[p][ix(b, f, r)] = face_m(b, ws.P, p, f, r);
    }
    const int c0 = max(cx0, 0), c1 = min(cx1, nx);
    for (int side = 0; side < 2; ++side) {  // south / north faces N(c, g)
      const int g = side ? ny : 0;
      if (g < ry0 || g > ry1) continue;
      for (int c = c0 + lane; c < c1; c += 32) b.N[p][ix(b, c, g)] = face_n(b, ws.P, p, c, g);
    }
  }
  if ((td.flags & kTfRing) && !(b.nest & kNestFull)) {
    const int c0 = max(cx0, 0), c1 = min(cx1, nx), r0 = max(ry0, 0), r1 = min(ry1, ny);
    for (int q = 0; q < b.child_count; ++q) {
      const Blk<T> ch = RTI_BLK(kp, RTI_KID(kp, b.child_first + q));
      const int a0 = ch.i0, a1 = ch.i0 + ch.nx / 3, b0 = ch.j0, b1 = ch.j0 + ch.ny / 3;
      // the footprint's inner ring within the region: rows b0 and b1-1 (all columns),
      // columns a0 and a1-1 (rows strictly between)
      const int hc0 = max(c0, a0), hc1 = min(c1, a1), nh = max(hc1 - hc0, 0);
      const int vr0 = max(r0, b0 + 1), vr1 = min(r1, b1 - 1), nv = max(vr1 - vr0, 0);
      const bool rb = b0 >= r0 && b0 < r1, rt = b1 - 1 >= r0 && b1 - 1 < r1 && b1 - 1 != b0;
      const bool cl = a0 >= c0 && a0 < c1, cr = a1 - 1 >= c0 && a1 - 1 < c1 && a1 - 1 != a0;
      const int n0 = rb ? nh : 0, n1 = rt ? nh : 0, n2 = cl ? nv : 0, n3 = cr ? nv : 0;
      for (int k = lane; k < n0 + n1 + n2 + n3; k += 32) {
        int I, J;
        if (k < n0) {
          I = hc0 + k;
          J = b0;
        } else if (k < n0 + n1) {
          I = hc0 + (k - n0);
          J = b1 - 1;
        } else if (k < n0 + n1 + n2) {
          I = a0;
          J = vr0 + (k - n0 - n1);
        } else {
          I = a1 - 1;
          J = vr0 + (k - n0 - n1 - n2);
        }
        const size_t o = ix(b, I, J);
        T rv;
        const bool wet = ring_patch(ch, b, p, I - a0, J - b0, b.h[o], rv);
        b.ring[o] = wet ? rv : ring_none(rv);
      }
    }
  }
  __syncwarp();
}

// Step strip td at chunk step s (one warp; ws holds the strip's staged descriptor, the
// prepass has run). The budget slot of the strip receives sum(eta^{n+1}) and adds the
// clip, outflow and ring terms.
template <class T, bool kTrack, bool kLim, bool kFb, bool kRg, class WS>
__device__ __forceinline__ void march_strip(const KParams<T>& kp, WS& ws, Tile td, int s) {
  constexpr int kRingD = RingD<T>::D;
  const int lane = threadIdx.x;
  const Blk<T>& b = ws.b;
  const ScenDev sc = ws.sc;
  const int p = (int)((sc.base + s) & 1), q = p ^ 1;
  const int sn = (int)(sc.base + s + 1);
  // the descriptor fields of the march, as locals
  const int nx = b.nx, ny = b.ny, pitch = b.pitch;
  const bool root = !b.is_child;
  const T dtdx = b.dtdx, eps = b.eps, g = b.g;
  const MomK<T> K = mom_consts(b);
  const T thr = b.thr;
  const T* etaP = b.eta[p];
  const T* Mp = b.M[p];
  const T* Np = b.N[p];
  const T* hh = b.h;
  const float* man = b.man;
  T* etaQ = b.eta[q];
  T* Mq = b.M[q];
  T* Nq = b.N[q];
  T* emax = b.emax;
  const bool ring_strip = (td.flags & kTfRing) != 0;
  T* vmax = b.vmax;  // tracked iff kTrack
  const unsigned full = 0xffffffffu;

  const int c = td.x0 - 2 + lane;                            // this lane's column (>= -2)
  const bool col_ok = c + kXOff < pitch;                     // inside the allocated row
  const bool own_col = lane >= 2 && lane < 2 + kStripW && c < nx;
  const bool fb_last = kFb && own_col && (c + 3) % 3 == 2;  // last column of a patch (R8)
  const bool col_x = c >= 1 && c <= nx - 1;  // x-face (c, .) is interior
  const bool col_y = c >= 0 && c <= nx - 1;  // y-face (c, .) lies on a cell column
  const int sl = (lane - 1) & 31, sr = (lane + 1) & 31;  // neighbour bit of a ballot
  const int y0 = td.y0, ye = min(y0 + kp.ty, ny);
  int fb_ph = (y0 + 1) % 3;  // row r mod 3, from row y0 - 2 (full-feedback march only)
  // this lane's budget partials over the strip's rows (state precision, branch-free
  // adds; the strip's sums are formed and scaled in binary64 at the end)
  T vol_t = T(0), clip_t = T(0), out_t = T(0), ring_t = T(0);
  const bool edge_strip = td.x0 == 0 || td.x0 + kStripW >= nx || y0 == 0 || ye == ny;
  // element offsets within a plane fit in 32 bits (rti_create checks pitch x rows < 2^31)
  int o = (y0 - 2 + kYOff) * pitch + (c + kXOff);

  // prologue: N^n of y-face (c, y0 - 2); rows y0 - 2 .. y0 + kRingD - 5 staged
  T nS = col_ok ? __ldcg(Np + o) : T(0);  // y0 - 2 is below row 0 or an interior row
  T nSL = __shfl_up_sync(full, nS, 1);
  const int x0 = td.x0;
  int rowbase = (y0 - 2 + kYOff) * pitch + x0;
  const StageLane SL = stage_lane<T>(lane, x0, pitch);
  for (int k = 0; k < kRingD - 2; ++k) {
    stage_row<T, kTrack>(ws.ring[k], etaP, hh, Mp, Np, emax, man, vmax,
                         kRg && ring_strip ? b.ring : nullptr, rowbase + k * pitch, pitch, SL,
                         y0 - 2 + k <= ye);
    cp_async_commit();
  }
  Row<T> A = {}, B = {}, C = {};
  T e_prev = T(0);  // eta^n of cell (c, r - 1) (velocity tracking only)

  // One row r from its inputs `cur`: X receives row r; Y, Z are rows r - 2, r - 1.
  auto row = [&](const Raw<T>& cur, Row<T>& X, const Row<T>& Y, const Row<T>& Z, int r) {
    const bool rin_x = r >= 0 && r <= ny - 1, rin_y = r >= 1 && r <= ny - 1;

    // ---- row r: eta^{n+1} (R1, R5, R7 pulls, R8 ring) and the output update (R9)
    Row<T> Nw;
    const T m = cur.m, nn = cur.nn;  // a child's edge faces hold the pulled fluxes
    Nw.H = cur.h;
    Nw.MX = m;
    Nw.NY = nS;
    Nw.nm = cur.nm;
    Nw.mE = __shfl_down_sync(full, m, 1);
    const T nnL = __shfl_up_sync(full, nn, 1);
    const bool own = own_col && r >= y0 && r < ye;
    if (kTrack) {  // R11: the state this step starts from (eta^n, M^n, N^n)
      // each face's velocity over that face's depth; a block edge's face has the edge
      // cell's depth (its neighbour taken as the cell itself)
      const T eW = __shfl_up_sync(full, cur.e, 1), hW = __shfl_up_sync(full, cur.h, 1);
      const T eE = __shfl_down_sync(full, cur.e, 1), hE = __shfl_down_sync(full, cur.h, 1);
      const bool w_in = c > 0, e_in = c < nx - 1, s_in = r > 0, n_in = r < ny - 1;
      const T Dw = T(0.5) * ((w_in ? hW : cur.h) + cur.h) + T(0.5) * ((w_in ? eW : cur.e) + cur.e);
      const T De = T(0.5) * (cur.h + (e_in ? hE : cur.h)) + T(0.5) * (cur.e + (e_in ? eE : cur.e));
      const T Ds = T(0.5) * ((s_in ? Z.H : cur.h) + cur.h) + T(0.5) * ((s_in ? e_prev : cur.e) + cur.e);
      const T Dn = T(0.5) * (cur.h + (n_in ? cur.hN : cur.h)) + T(0.5) * (cur.e + (n_in ? cur.eN : cur.e));
      const T D = cur.h + cur.e;
      if (own && D > eps) {
        const T u = T(0.5) * (Ar<T>::face_vel(m, Dw, eps) + Ar<T>::face_vel(Nw.mE, De, eps));
        const T v = T(0.5) * (Ar<T>::face_vel(nS, Ds, eps) + Ar<T>::face_vel(nn, Dn, eps));
        const T s2 = u * u + v * v;
        if (s2 > cur.vm) vmax[o] = s2;
      }
      e_prev = cur.e;
    }
    T e = cur.e - (dtdx * (Nw.mE - m) + dtdx * (nn - nS));
    const bool clipped = Nw.H + e < T(0);
    clip_t += (clipped && own) ? -Nw.H - e : T(0);
    e = clipped ? -Nw.H : e;
    if constexpr (kFb) {  // full feedback: this block's own level, and the patches row r completes
      ws.fb[fb_ph][lane] = e;  // each lane keeps its own column: no barrier needed
      if (fb_ph == 2 && r >= y0 && r < ye)
        patch_means(b, ws.P, ws.fb[0][lane], Y.H, ws.fb[1][lane], Z.H, e, Nw.H, fb_last, c, r);
      fb_ph = fb_ph == 2 ? 0 : fb_ph + 1;
    }
    if (ring_strip) {  // fine-to-coarse override (R8), formed by the prepass
      const T rv = !col_ok ? ring_none(T(0)) : kRg ? cur.rv : __ldcg(b.ring + o);
      if (!ring_unset(rv) && col_y && rin_x) {
        ring_t += own ? rv - e : T(0);
        e = rv;
      }
    }
    Nw.E = e;
    {  // output update (predicated stores, no branches)
      const T em = cur.em;
      const bool up = own && Nw.H + e > eps && e > em;
      const bool arrives = up && em < thr && e >= thr;
      if (own) etaQ[o] = e;
      if (up) emax[o] = e;
      if (arrives) b.arr[o] = sn;
      vol_t += own ? e : T(0);  // a non-finite level makes the strip's sum non-finite
    }
    if (edge_strip) {  // flux through the block's edges (outflow positive)
      T of = T(0);
      of -= (own && c == 0) ? m : T(0);
      of += (own && c == nx - 1) ? Nw.mE : T(0);
      of -= (own && r == 0) ? nS : T(0);
      of += (own && r == ny - 1) ? nn : T(0);
      out_t += of;
    }

    // ---- advective face terms of row r
    Nw.eL = __shfl_up_sync(full, e, 1);
    Nw.hL = __shfl_up_sync(full, Nw.H, 1);
    unsigned fx;
    {  // x-face (c, r)
      const T dep = T(0.5) * (Nw.hL + Nw.H) + T(0.5) * (Nw.eL + Nw.E);
      const bool in = col_x && rin_x;
      fx = (in && dep > eps) ? 1u : 0u;
      Nw.nb = T(0.25) * ((nSL + nS) + (nnL + nn));
      // Binary32 divides everywhere: a face without a usable depth gets a value that
      // every reader masks (usable flags) or discards (no wet pair on its own face).
      T qx = T(0), rx = T(0);
      if (Ar<T>::kSelect || (in && dep != T(0))) Ar<T>::quot2(m * m, m * Nw.nb, dep, qx, rx);
      Nw.QX = qx;
      Nw.RX = rx;
    }
    {  // y-face (c, r)
      const T dep = T(0.5) * (Z.H + Nw.H) + T(0.5) * (Z.E + Nw.E);
      const bool in = col_y && rin_y;
      Nw.fl = fx | ((in && dep > eps) ? 2u : 0u);
      Nw.mb = T(0.25) * ((Z.MX + m) + (Z.mE + Nw.mE));
      T sy = T(0), ty = T(0);
      if (Ar<T>::kSelect || (in && dep != T(0))) Ar<T>::quot2(nS * nS, nS * Nw.mb, dep, sy, ty);
      Nw.SY = sy;
      Nw.TY = ty;
    }
    X = Nw;
    nS = nn;
    nSL = nnL;

    // ---- row j = r - 1 (rows Y, Z, X = j-1, j, j+1): M^{n+1}, N^{n+1} (R2-R4), root edges (R6)
    if (r > y0) {
      const int j = r - 1;
      // a warp whose cells on both sides of every owned face are dry updates nothing;
      // one whose owned faces are all in open water takes the short form
      const bool wA = Y.H + Y.E > eps, wB = Z.H + Z.E > eps, wW = Z.hL + Z.eL > eps;
      const bool act = own_col && (wW || wB || wA);
      // open water for the whole warp: the faces of lanes 1..30 (the owned lanes and
      // their neighbours) are usable and every owned face has wet cells on both sides
      const bool open = lane == 0 || lane == 31 ||
                        (Z.fl == 3u && (!own_col || (wW && wB && wA && (Y.fl & X.fl) == 3u)));
      T xm = T(0), ym = T(0);
      if (__all_sync(full, open)) {
        const T qm = __shfl_up_sync(full, Z.QX, 1), qp = __shfl_down_sync(full, Z.QX, 1);
        const T tw = __shfl_up_sync(full, Z.TY, 1), te = __shfl_down_sync(full, Z.TY, 1);
        const float nmL = __shfl_up_sync(full, Z.nm, 1);
        xm = mom_open<kLim>(Z.hL, Z.eL, Z.H, Z.E, Z.MX, Z.nb, qm, Z.QX, qp, Y.RX, Z.RX, X.RX, nmL,
                      Z.nm, K);
        ym = mom_open<kLim>(Y.H, Y.E, Z.H, Z.E, Z.NY, Z.mb, Y.SY, Z.SY, X.SY, tw, Z.TY, te, Y.nm,
                      Z.nm, K);
      } else if (__any_sync(full, act)) {
        const T qm = __shfl_up_sync(full, Z.QX, 1), qp = __shfl_down_sync(full, Z.QX, 1);
        const T tw = __shfl_up_sync(full, Z.TY, 1), te = __shfl_down_sync(full, Z.TY, 1);
        const float nmL = __shfl_up_sync(full, Z.nm, 1);
        const unsigned bx = __ballot_sync(full, Z.fl & 1u), by = __ballot_sync(full, Z.fl & 2u);
        xm = xmom_r<kLim>(Z.hL, Z.eL, Z.H, Z.E, Z.MX, Z.nb, ((bx >> sl) & 1u) != 0, qm, Z.QX,
                    ((bx >> sr) & 1u) != 0, qp, (Y.fl & 1u) != 0, Y.RX, Z.RX, (X.fl & 1u) != 0,
                    X.RX, nmL, Z.nm, K);
        ym = ymom_r<kLim>(Y.H, Y.E, Z.H, Z.E, Z.NY, Z.mb, (Y.fl & 2u) != 0, Y.SY, Z.SY,
                    (X.fl & 2u) != 0, X.SY, ((by >> sl) & 1u) != 0, tw, Z.TY,
                    ((by >> sr) & 1u) != 0, te, Y.nm, Z.nm, K);
      }
      if (!edge_strip) {  // interior strip: every owned face is an interior face
        if (own_col) {
          Mq[o - pitch] = xm;
          Nq[o - pitch] = ym;
        }
      } else if (own_col) {
        const int oj = o - pitch;
        if (c >= 1) Mq[oj] = xm;
        else if (root) Mq[oj] = b.bc[0] == kBcRadiation ? radiate_r(Z.H, Z.E, T(-1), eps, g) : T(0);
        if (c == nx - 1 && root)
          Mq[oj + 1] = b.bc[1] == kBcRadiation ? radiate_r(Z.H, Z.E, T(1), eps, g) : T(0);
        if (j >= 1) Nq[oj] = ym;
        else if (root) Nq[oj] = b.bc[2] == kBcRadiation ? radiate_r(Z.H, Z.E, T(-1), eps, g) : T(0);
        if (j == ny - 1 && root)
          Nq[oj + pitch] = b.bc[3] == kBcRadiation ? radiate_r(Z.H, Z.E, T(1), eps, g) : T(0);
      }
    }
    o += pitch;
  };

  int slot = 0;  // ring slot of row r
  for (int r = y0 - 2; r <= ye; ++r) {
    // refill the slot of row r - 2: every lane read it before the __syncwarp of row r - 1
    stage_row<T, kTrack>(ws.ring[(slot - 2) & (kRingD - 1)], etaP, hh, Mp, Np, emax, man,
                         vmax, kRg && ring_strip ? b.ring : nullptr,
                         rowbase + (kRingD - 2) * pitch,
                         pitch, SL, r + kRingD - 2 <= ye);
    cp_async_commit();
    if (kTrack) cp_async_wait<kRingD - 3>();  // rows r and r + 1 have landed
    else cp_async_wait<kRingD - 2>();         // row r has landed
    __syncwarp();                             // ... for every lane's chunks
    Raw<T> cur = read_row<T, kTrack>(ws.ring[slot], lane);
    if constexpr (kRg) {
      if (ring_strip) cur.rv = ws.ring[slot].rg[lane + 2];
    }
    if (kTrack) {
      const auto& nx1 = ws.ring[(slot + 1) & (kRingD - 1)];
      cur.eN = nx1.e[lane + 2];
      cur.hN = nx1.h[lane + 2];
    }
    slot = (slot + 1) & (kRingD - 1);
    rowbase += pitch;
    Row<T> X;
    row(cur, X, B, C, r);
    A = B;  // rows r-2, r-1, r
    B = C;
    C = X;
  }

  cp_async_wait<0>();  // (only empty groups can be outstanding here)
  __syncwarp();

  // ---- the strip's budget partials (binary64, fixed reduction order)
  const double vs = warp_sum((double)vol_t);
  if (lane == 0 && !dfinite(vs)) atomicOr(b.status, kStNonFinite);
  const double cs = warp_sum((double)clip_t) * b.dx2, os = warp_sum((double)out_t) * b.vol,
               rs = warp_sum((double)ring_t) * b.dx2;
  if (lane == 0) {
    double* slot = b.budget + 4 * (size_t)((y0 / kp.ty) * b.tiles_x + td.x0 / kp.tx);
    slot[0] = vs;
    slot[1] += cs;
    slot[2] += os;
    slot[3] += rs;
  }
}

// ------------------------------------------------------------------ device-wide barrier

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
// Steps [s_first, s_first + s_count) of a chunk over every strip of the work list (the
// kStepTrack variant also carries the maximum-velocity update, for groups that need it).
// The warps take strips from a device counter per step (heavy strips come first in the
// list), so a slow strip delays no fixed set of others. Counter s & 1 serves step s;
// the other one is cleared during step s, when no warp can still be taking from it
// (step s - 1 has ended: a barrier or the previous launch lies between). With more than
// one step the launch must be cooperative: consecutive steps are separated by the
// device-wide barrier. Variants (kMode): kStepPlain; kStepTrack, whose strips of blocks
// that keep the maximum velocity take the tracking march. The flag kStepLimit added to a
// variant compiles in the velocity limit (a block without it has vlim = +inf, so its
// fluxes are unchanged); groups without the limit run variants that do not evaluate it
// at all. The flag kStepFull selects k_step_flow, which compiles in full feedback: the
// strips of a child with it march with patch_means, which forms the parent's 3x3 means
// from the levels in registers, and each sets its flag in kp.done once its step has been
// stored; the parent's ring strips wait for the flags of the child strips under their
// region (wait_ring_means). A flag holds the last step of the chunk its strip has ended
// (cleared at the chunk's start). With more than one step k_step_flow runs the chunk as
// one dataflow: every strip sets its flag, and a strip's next step waits only for the
// strips it depends on (the host's lists, dataflow_deps) instead of a device-wide
// barrier, so the end of one step overlaps the start of the next.
// Resident CTAs per SM the register allocation targets: binary32 fits 96 registers
// (5 CTAs of 4 warps) with at most a few spilled words; its variants with full feedback
// or velocity tracking, which spilled 36-100 B at that cap and ran 8-12 % slower, take
// 128 (4 CTAs); binary64 keeps the compiler's choice.
template <class T, int kMode>
struct StepOcc {
  static constexpr int kMinBlocks = 1;
};
template <int kMode>
struct StepOcc<float, kMode> {
  static constexpr int kMinBlocks = (kMode & (kStepFull | kStepTrack)) ? 4 : 5;
};

// One strip t at chunk step s: its prepass, its full-feedback wait, its march, and its
// flag where a strip waits on it (full feedback, or the dataflow `df` of a full-feedback
// group, where it first waits for the strips it depends on to end step s - 1).
template <class T, int kMode, class WS>
__device__ __forceinline__ void strip_step(const KParams<T>& kp, WS& ws, int t, int s,
                                           int s_first, bool df, const int* dep_idx) {
  constexpr bool kAnyTrack = (kMode & kStepTrack) != 0;
  constexpr bool kLim = (kMode & kStepLimit) != 0;
  constexpr bool kAnyFull = (kMode & kStepFull) != 0;
  const Tile td = kp.tiles[t];
  stage_strip(kp, ws, td.blk);
  if ((long long)s >= ws.sc.remaining) return;  // the scenario has finished
  if constexpr (kAnyFull) {
    if (df && s > s_first)  // the strips this one depends on have ended step s - 1
      wait_flags(kp, dep_idx + kp.dep_off[t], kp.dep_off[t + 1] - kp.dep_off[t],
                 ((unsigned long long)(s - 1) << 32) | kDoneAll);
  }
  if ((td.flags & kTfRing) || ws.b.is_child)
    strip_prepass(kp, ws, td, (int)((ws.sc.base + s) & 1));
  if constexpr (kAnyFull) {  // a parent's ring strip: its children's means of step s
    if ((td.flags & kTfRing) && (ws.b.nest & kNestFull)) wait_ring_means(kp, ws, td, s);
    const bool fb = ws.b.is_child && (ws.b.nest & kNestFull);
    if (kAnyTrack && ws.b.vmax) {  // velocity tracked; the ring plane staged (kRg)
      if (fb) march_strip<T, true, kLim, true, true>(kp, ws, td, s);
      else march_strip<T, true, kLim, false, true>(kp, ws, td, s);
    } else {
      if (fb) march_strip<T, false, kLim, true, true>(kp, ws, td, s);
      else march_strip<T, false, kLim, false, true>(kp, ws, td, s);
    }
    if (fb || df)
      strip_finished(kp.done + ws.b.strip0 + (td.y0 / kp.ty) * ws.b.tiles_x + td.x0 / kp.tx, s);
  } else {
    if (kAnyTrack && ws.b.vmax) march_strip<T, true, kLim, false, false>(kp, ws, td, s);
    else march_strip<T, false, kLim, false, false>(kp, ws, td, s);
  }
}

template <class T, int kMode>
__global__ void __launch_bounds__(kWarps * 32, StepOcc<T, kMode>::kMinBlocks)
    k_step(KParams<T> kp, int s_first, int s_count) {
  constexpr bool kAnyTrack = (kMode & kStepTrack) != 0;
  constexpr bool kLim = (kMode & kStepLimit) != 0;  // some block keeps the velocity limit
  static_assert((kMode & kStepFull) == 0, "the full-feedback variants run k_step_flow");
  __shared__ WarpSlot<T, false> slots[kWarps];
  __shared__ int go;
  WarpSlot<T, false>& ws = slots[threadIdx.y];
  if (threadIdx.x == 0) ws.blk = -1;
  __syncwarp();
  unsigned gen = 0;
  if (s_count > 1 && threadIdx.x == 0 && threadIdx.y == 0) gen = ld_acquire_u32(&kp.bar->gen);
  const int nt = *kp.ntiles;
  for (int s = s_first; s < s_first + s_count; ++s) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0)
      atomicExch(&kp.bar->next[(s + 1) & 1], 0u);
    for (;;) {
      unsigned t = 0;
      if (threadIdx.x == 0) t = atomicAdd(&kp.bar->next[s & 1], 1u);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t >= (unsigned)nt) break;
      const Tile td = kp.tiles[t];
      stage_strip(kp, ws, td.blk);
      if ((long long)s >= ws.sc.remaining) continue;  // the scenario has finished
      if ((td.flags & kTfRing) || ws.b.is_child)
        strip_prepass(kp, ws, td, (int)((ws.sc.base + s) & 1));
      if (kAnyTrack && ws.b.vmax) march_strip<T, true, kLim, false, false>(kp, ws, td, s);
      else march_strip<T, false, kLim, false, false>(kp, ws, td, s);
    }
    if (s + 1 < s_first + s_count &&
        !grid_barrier(kp.bar, gen, kp.status, kp.spin_cycles, &go))
      return;
  }
}

// The step kernel of full-feedback groups (kMode has kStepFull): the same strips, but a
// chunk runs as one dataflow when its dependency lists are given (kp.dep_off).
template <class T, int kMode>
__global__ void __launch_bounds__(kWarps * 32, StepOcc<T, kMode>::kMinBlocks)
    k_step_flow(KParams<T> kp, int s_first, int s_count) {
  static_assert((kMode & kStepFull) != 0, "the full-feedback variants");
  __shared__ WarpSlot<T, true> slots[kWarps];
  __shared__ int go;
  WarpSlot<T, true>& ws = slots[threadIdx.y];
  if (threadIdx.x == 0) ws.blk = -1;
  __syncwarp();
  const int nt = *kp.ntiles;
  unsigned gen = 0;
  {
    // A chunk of a full-feedback group runs as one dataflow: its steps x strips in one
    // sequence, each strip starting once the strips it depends on have ended the previous
    // step (no device-wide barrier, so a step's end overlaps the next step's start).
    const bool df = kp.dep_off && s_count > 1 &&
                    (unsigned long long)s_count * (unsigned long long)nt < 0xff000000ull;
    const unsigned total = df ? (unsigned)s_count * (unsigned)nt : 0u;
    const int* dep_idx = df ? kp.dep_off + nt + 1 : nullptr;
    if (!df && s_count > 1 && threadIdx.x == 0 && threadIdx.y == 0)
      gen = ld_acquire_u32(&kp.bar->gen);
    int s = s_first;
    if (!df && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0)
      atomicExch(&kp.bar->next[(s + 1) & 1], 0u);
    for (;;) {
      unsigned i = 0;
      if (threadIdx.x == 0) i = atomicAdd(&kp.bar->next[df ? 0 : (s & 1)], 1u);
      i = __shfl_sync(0xffffffffu, i, 0);
      int t;
      if (df) {
        if (i >= total) break;
        s = s_first + (int)(i / (unsigned)nt);
        t = (int)(i % (unsigned)nt);
      } else {
        if (i >= (unsigned)nt) {  // this step's strips are all taken
          if (s + 1 >= s_first + s_count) break;
          if (!grid_barrier(kp.bar, gen, kp.status, kp.spin_cycles, &go)) return;
          ++s;
          if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0)
            atomicExch(&kp.bar->next[(s + 1) & 1], 0u);
          continue;
        }
        t = (int)i;
      }
      strip_step<T, kMode>(kp, ws, t, s, s_first, df, dep_idx);
    }
  }
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
