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
//     and the outflow limit; radiation or wall faces on root edges.
//
// eta, M and N are ping-ponged (parity = step & 1), so no pass reads what it writes
// and every pull reads a time level that no tile of the same pass modifies.
// The discrete rules follow the oracle's readings R1-R10 operation for operation;
// the binary64 build uses -fmad=false so that it rounds like the oracle.
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
#define RTI_IX(c, r, pitch, ny, code) checked_ix((c), (r), (pitch), (ny), (code))
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
#define RTI_BLK(kp, i) (kp).blk[checked_idx((i), (kp).nblk, 10)]
template <class B>
__device__ __forceinline__ void check_ptr(const B& b, const void* p, int code) {
  if ((const char*)p < b.lo || (const char*)p >= b.hi) {
    if (atomicCAS(&g_rti_check[0], 0, code) == 0) {
      g_rti_check[5] = blockIdx.x;
      g_rti_check[6] = (int)((const char*)p - b.lo);
      g_rti_check[7] = b.nx;
    }
  }
}
#define RTI_CHKP(b, p, code) check_ptr((b), (p), (code))
#define RTI_KID(kp, i) (kp).kids[checked_idx((i), (kp).nkids, 11)]
#else
#define RTI_IX(c, r, pitch, ny, code) ((size_t)((r) + kYOff) * (size_t)(pitch) + (size_t)((c) + kXOff))
#define RTI_BLK(kp, i) (kp).blk[(i)]
#define RTI_CHKP(b, p, code) ((void)0)
#define RTI_KID(kp, i) (kp).kids[(i)]
#endif

template <class T>
__device__ __forceinline__ size_t ix(const Blk<T>& b, int c, int r) {
  return RTI_IX(c, r, b.pitch, b.ny, 1);
}

// ------------------------------------------------------------------ coarse -> fine (R7)
// Fine face t of an edge whose coarse faces are v(k), k = 0..K-1: the coarse value at
// the middle fine face, (2 v_k + v_{k+-1}) / 3 at the outer ones, neighbour clamped.
template <class T>
__device__ __forceinline__ T edge_interp(const T* arr, const Blk<T>& P, int fixed, int start,
                                         int K, int t, bool along_y) {
  int k = t / 3, sub = t - 3 * k;
  double vk = along_y ? (double)arr[ix(P, fixed, start + k)] : (double)arr[ix(P, start + k, fixed)];
  if (sub == 1) return (T)vk;
  int kn = sub == 0 ? k - 1 : k + 1;
  kn = kn < 0 ? 0 : (kn > K - 1 ? K - 1 : kn);
  double vn = along_y ? (double)arr[ix(P, fixed, start + kn)] : (double)arr[ix(P, start + kn, fixed)];
  return (T)((2.0 * vk + vn) / 3.0);
}

// x-flux of face (f, j) at parity p; a child's edge faces come from the parent.
template <class T>
__device__ __forceinline__ T face_m(const KParams<T>& kp, const Blk<T>& b, int p, int f, int j) {
  if (b.is_child && (f == 0 || f == b.nx)) {
#ifdef RTI_CHECKED
    if (b.parent < 0 && atomicCAS(&g_rti_check[0], 0, 3) == 0) g_rti_check[5] = blockIdx.x;
#endif
    const Blk<T>& P = RTI_BLK(kp, b.parent);
    int F = b.i0 + (f == 0 ? 0 : b.nx / 3);
    return edge_interp<T>(P.M[p], P, F, b.j0, b.ny / 3, j, true);
  }
  return b.M[p][ix(b, f, j)];
}
template <class T>
__device__ __forceinline__ T face_n(const KParams<T>& kp, const Blk<T>& b, int p, int i, int g) {
  if (b.is_child && (g == 0 || g == b.ny)) {
    const Blk<T>& P = RTI_BLK(kp, b.parent);
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

// eta^{n+1} of child cell (x, y) recomputed from the child's stable level p
template <class T>
__device__ T child_eta_next(const KParams<T>& kp, const Blk<T>& c, int p, int x, int y) {
  T Mw = face_m(kp, c, p, x, y), Me = face_m(kp, c, p, x + 1, y);
  T Ns = face_n(kp, c, p, x, y), Nn = face_n(kp, c, p, x, y + 1);
  double dummy = 0.0;
  return mass(c, p, x, y, Mw, Me, Ns, Nn, dummy);
}

// ------------------------------------------------------------------ fine -> coarse (R8)
// If parent cell (I, J) lies on the inner ring of a child footprint and the 3x3 patch
// has a wet cell, store the floored mean of the wet child levels in `out`.
template <class T>
__device__ bool ring_value(const KParams<T>& kp, const Blk<T>& b, int p, int I, int J, T hP,
                           T& out) {
  for (int q = 0; q < b.child_count; ++q) {
    const Blk<T>& c = RTI_BLK(kp, RTI_KID(kp, b.child_first + q));
    int a = c.nx / 3, bb = c.ny / 3;
    int u = I - c.i0, v = J - c.j0;
    if (u < 0 || v < 0 || u >= a || v >= bb) continue;
    if (!(u == 0 || u == a - 1 || v == 0 || v == bb - 1)) return false;
    double sum = 0.0;
    int wet = 0;
    for (int x = 3 * u; x < 3 * u + 3; ++x) {    // outer: x (the paper's J)
      for (int y = 3 * v; y < 3 * v + 3; ++y) {  // inner: y (the paper's I)
        T e = child_eta_next(kp, c, p, x, y);
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
struct Fld {
  const T* e;  // eta^{n+1}
  const T* h;
  const T* M;  // M^n
  const T* N;  // N^n
  const float* n;
  int pitch, nx, ny;
  T eps;
  __device__ __forceinline__ size_t at(int c, int r) const { return RTI_IX(c, r, pitch, ny, 2); }
  __device__ __forceinline__ T dep_x(int f, int j) const {
    size_t L = at(f - 1, j), R = at(f, j);
    return T(0.5) * (h[L] + h[R]) + T(0.5) * (e[L] + e[R]);
  }
  __device__ __forceinline__ T dep_y(int i, int g) const {
    size_t S = at(i, g - 1), Nc = at(i, g);
    return T(0.5) * (h[S] + h[Nc]) + T(0.5) * (e[S] + e[Nc]);
  }
  __device__ __forceinline__ bool ok_x(int f, int j) const {
    return f >= 1 && f <= nx - 1 && j >= 0 && j <= ny - 1 && dep_x(f, j) > eps;
  }
  __device__ __forceinline__ bool ok_y(int i, int g) const {
    return g >= 1 && g <= ny - 1 && i >= 0 && i <= nx - 1 && dep_y(i, g) > eps;
  }
  __device__ __forceinline__ T nbar_x(int f, int j) const {
    return T(0.25) * ((N[at(f - 1, j)] + N[at(f, j)]) + (N[at(f - 1, j + 1)] + N[at(f, j + 1)]));
  }
  __device__ __forceinline__ T mbar_y(int i, int g) const {
    return T(0.25) * ((M[at(i, g - 1)] + M[at(i, g)]) + (M[at(i + 1, g - 1)] + M[at(i + 1, g)]));
  }
  __device__ __forceinline__ T qx(int f, int j) const {
    T m = M[at(f, j)];
    return (m * m) / dep_x(f, j);
  }
  __device__ __forceinline__ T rx(int f, int j) const {
    return (M[at(f, j)] * nbar_x(f, j)) / dep_x(f, j);
  }
  __device__ __forceinline__ T qy(int i, int g) const {
    T v = N[at(i, g)];
    return (v * v) / dep_y(i, g);
  }
  __device__ __forceinline__ T ry(int i, int g) const {
    return (N[at(i, g)] * mbar_y(i, g)) / dep_y(i, g);
  }
};

template <class T>
__device__ __forceinline__ T upwind(T w, T phim, T phi0, T phip, bool okm, bool okp) {
  if (w > T(0)) return okm ? phi0 - phim : T(0);
  if (w < T(0)) return okp ? phip - phi0 : T(0);
  return (okm && okp) ? T(0.5) * (phip - phim) : T(0);
}

template <class T>
__device__ __forceinline__ T flux_update(const Blk<T>& b, T m, T across, T Df, T grad, T adv,
                                         T nf) {
  T P = b.g * Df * b.dtdx * grad;
  T F = b.cfric * nf * nf * dsqrt(m * m + across * across) / (Df * Df * dcbrt(Df));
  return ((T(1) - F) * m - adv - P) / (T(1) + F);
}

template <class T>
__device__ __forceinline__ T limit_outflow(T m, T Dlo, T Dhi, T dx, T q4dt) {
  T cap = (m > T(0) ? Dlo : Dhi) * dx / q4dt;
  if (m > cap) return cap;
  if (m < -cap) return -cap;
  return m;
}

template <class T>
__device__ T xmom(const Blk<T>& b, const Fld<T>& F, int f, int j) {
  const T eps = b.eps;
  size_t L = F.at(f - 1, j), R = F.at(f, j);
  T eL = F.e[L], eR = F.e[R], hL = F.h[L], hR = F.h[R];
  bool wL = hL + eL > eps, wR = hR + eR > eps;
  T m = F.M[R];
  T Df, grad, adv;
  if (wL && wR) {
    Df = T(0.5) * (hL + hR) + T(0.5) * (eL + eR);
    grad = eR - eL;
    bool okm = F.ok_x(f - 1, j), okp = F.ok_x(f + 1, j);
    T ax = upwind(m, okm ? F.qx(f - 1, j) : T(0), F.qx(f, j), okp ? F.qx(f + 1, j) : T(0), okm,
                  okp);
    T nb = F.nbar_x(f, j);
    bool oks = F.ok_x(f, j - 1), okn = F.ok_x(f, j + 1);
    T ay = upwind(nb, oks ? F.rx(f, j - 1) : T(0), F.rx(f, j), okn ? F.rx(f, j + 1) : T(0), oks,
                  okn);
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
  float nL = F.n[L], nR = F.n[R];
  T nf = (T)(nL > nR ? nL : nR);
  T m1 = flux_update(b, m, F.nbar_x(f, j), Df, grad, adv, nf);
  if (!(wL && wR) && (wL ? m1 < T(0) : m1 > T(0))) return T(0);
  return limit_outflow(m1, hL + eL, hR + eR, b.dx, b.q4dt);
}

template <class T>
__device__ T ymom(const Blk<T>& b, const Fld<T>& F, int i, int g) {
  const T eps = b.eps;
  size_t S = F.at(i, g - 1), Nc = F.at(i, g);
  T eS = F.e[S], eN = F.e[Nc], hS = F.h[S], hN = F.h[Nc];
  bool wS = hS + eS > eps, wN = hN + eN > eps;
  T v = F.N[Nc];
  T Df, grad, adv;
  if (wS && wN) {
    Df = T(0.5) * (hS + hN) + T(0.5) * (eS + eN);
    grad = eN - eS;
    bool okm = F.ok_y(i, g - 1), okp = F.ok_y(i, g + 1);
    T ay = upwind(v, okm ? F.qy(i, g - 1) : T(0), F.qy(i, g), okp ? F.qy(i, g + 1) : T(0), okm,
                  okp);
    T mb = F.mbar_y(i, g);
    bool okw = F.ok_y(i - 1, g), oke = F.ok_y(i + 1, g);
    T ax = upwind(mb, okw ? F.ry(i - 1, g) : T(0), F.ry(i, g), oke ? F.ry(i + 1, g) : T(0), okw,
                  oke);
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
  float nS = F.n[S], nN = F.n[Nc];
  T nf = (T)(nS > nN ? nS : nN);
  T v1 = flux_update(b, v, F.mbar_y(i, g), Df, grad, adv, nf);
  if (!(wS && wN) && (wS ? v1 < T(0) : v1 > T(0))) return T(0);
  return limit_outflow(v1, hS + eS, hN + eN, b.dx, b.q4dt);
}

// R6: flux leaving through a root edge next to cell c (sign +1 east/north, -1 west/south)
template <class T>
__device__ __forceinline__ T radiate(const Blk<T>& b, const Fld<T>& F, size_t c, T sign) {
  T h = F.h[c], e = F.e[c];
  if (!(h + e > b.eps)) return T(0);
  return sign * (dsqrt(b.g * (h > T(0) ? h : T(0))) * e);
}

// ------------------------------------------------------------------ block reduction
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ tiles
// Note on descriptors: each tile copies its block descriptor once instead of
// re-reading its fields through a reference into the device table. With references,
// optimised binary64 builds faulted on an edge-row read whose index and pointer were
// both verified in range by the range-checked build; the unoptimised (-G) build and
// the copied-descriptor form never did. The mixed-sequence GPU test guards this.
// CTA of 32 x 8 threads; each thread walks the tile in steps of (32, 8).
template <class T>
__device__ void pass_a_tile(const KParams<T>& kp, int t, int s, double (*red)[8]) {
  const Tile td = kp.tiles[t];
  const Blk<T> b = RTI_BLK(kp, td.blk);  // copied: see the note on descriptors
  const ScenDev sc = kp.scen[b.scen];
  if ((long long)s >= sc.remaining) return;  // uniform over the CTA
  const int p = (int)((sc.base + s) & 1), q = p ^ 1;
  const int sn = (int)(sc.base + s + 1);
  double vol = 0.0, clip = 0.0, out = 0.0, ring = 0.0;
  bool bad = false;
  const int xe = min(td.x0 + kp.tx, b.nx), ye = min(td.y0 + kp.ty, b.ny);
  for (int j = td.y0 + threadIdx.y; j < ye; j += 8) {
    for (int i = td.x0 + threadIdx.x; i < xe; i += 32) {
      T Mw = face_m(kp, b, p, i, j), Me = face_m(kp, b, p, i + 1, j);
      T Ns = face_n(kp, b, p, i, j), Nn = face_n(kp, b, p, i, j + 1);
      if (b.is_child) {  // store the pulled edge fluxes for pass B
        RTI_CHKP(b, &b.M[p][ix(b, b.nx, j)], 24);
        RTI_CHKP(b, &b.N[p][ix(b, i, b.ny)], 25);
        if (i == 0) b.M[p][ix(b, 0, j)] = Mw;
        if (i == b.nx - 1) b.M[p][ix(b, b.nx, j)] = Me;
        if (j == 0) b.N[p][ix(b, i, 0)] = Ns;
        if (j == b.ny - 1) b.N[p][ix(b, i, b.ny)] = Nn;
      }
      double clip_c = 0.0;
      T e = mass(b, p, i, j, Mw, Me, Ns, Nn, clip_c);
      clip += clip_c;
      const size_t c = ix(b, i, j);
      const T h = b.h[c];
      if (td.flags & kTfRing) {
        T rv;
        if (ring_value(kp, b, p, i, j, h, rv)) {
          ring += ((double)rv - (double)e) * b.dx2;
          e = rv;
        }
      }
      RTI_CHKP(b, &b.eta[q][c], 20);
      RTI_CHKP(b, &b.emax[c], 21);
      RTI_CHKP(b, &b.arr[c], 22);
      b.eta[q][c] = e;
      T em = b.emax[c];
      if (h + e > b.eps && e > em) {
        if (em < b.thr && e >= b.thr) b.arr[c] = sn;
        b.emax[c] = e;
      }
      vol += (double)e;
      if (i == 0) out += b.vol * (double)(-Mw);
      if (i == b.nx - 1) out += b.vol * (double)Me;
      if (j == 0) out += b.vol * (double)(-Ns);
      if (j == b.ny - 1) out += b.vol * (double)Nn;
      bad |= !dfinite(e);
    }
  }
  if (bad) atomicOr(b.status, kStNonFinite);
  // per-tile binary64 budget: warp shuffles, then the 8 warps through shared memory
  vol = warp_sum(vol);
  clip = warp_sum(clip);
  out = warp_sum(out);
  ring = warp_sum(ring);
  const int w = threadIdx.y;
  if (threadIdx.x == 0) {
    red[0][w] = vol;
    red[1][w] = clip;
    red[2][w] = out;
    red[3][w] = ring;
  }
  __syncthreads();
  if (threadIdx.y == 0 && threadIdx.x < 4) {
    double a = 0.0;
    for (int k = 0; k < 8; ++k) a += red[threadIdx.x][k];
    double* slot = b.budget + 4 * (size_t)((td.y0 / kp.ty) * b.tiles_x + td.x0 / kp.tx);
    RTI_CHKP(b, slot + 3, 23);
    if (threadIdx.x == 0) slot[0] = a;
    else slot[threadIdx.x] += a;
  }
  __syncthreads();
}

template <class T>
__device__ void pass_b_tile(const KParams<T>& kp, int t, int s) {
  const Tile td = kp.tiles[t];
  const Blk<T> b = RTI_BLK(kp, td.blk);  // copied: see the note on descriptors
  const ScenDev sc = kp.scen[b.scen];
  if ((long long)s >= sc.remaining) return;
  const int p = (int)((sc.base + s) & 1), q = p ^ 1;
  Fld<T> F{b.eta[q], b.h, b.M[p], b.N[p], b.man, b.pitch, b.nx, b.ny, b.eps};
  T* Mo = b.M[q];
  T* No = b.N[q];
  const int xe = min(td.x0 + kp.tx, b.nx), ye = min(td.y0 + kp.ty, b.ny);
  const bool root = !b.is_child;
  for (int j = td.y0 + threadIdx.y; j < ye; j += 8) {
    for (int i = td.x0 + threadIdx.x; i < xe; i += 32) {
      // x-face i (west face of cell i), plus the east edge face
      RTI_CHKP(b, &Mo[F.at(i, j)], 30);
      RTI_CHKP(b, &No[F.at(i, j)], 31);
      RTI_CHKP(b, &F.e[F.at(i, j)], 32);
      RTI_CHKP(b, &F.M[F.at(i + 1, j + 1)], 33);
      if (i >= 1) {
        Mo[F.at(i, j)] = xmom(b, F, i, j);
      } else if (root) {
        Mo[F.at(0, j)] = b.bc[0] == kBcRadiation ? radiate(b, F, F.at(0, j), T(-1)) : T(0);
      }
      if (i == b.nx - 1 && root)
        Mo[F.at(b.nx, j)] = b.bc[1] == kBcRadiation ? radiate(b, F, F.at(i, j), T(1)) : T(0);
      // y-face j (south face of cell row j), plus the north edge face
      if (j >= 1) {
        No[F.at(i, j)] = ymom(b, F, i, j);
      } else if (root) {
        No[F.at(i, 0)] = b.bc[2] == kBcRadiation ? radiate(b, F, F.at(i, 0), T(-1)) : T(0);
      }
      if (j == b.ny - 1 && root)
        No[F.at(i, b.ny)] = b.bc[3] == kBcRadiation ? radiate(b, F, F.at(i, j), T(1)) : T(0);
    }
  }
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
                                             long long spin_cycles) {
  __shared__ int s_go;
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
    s_go = ok && !(*(volatile int*)status & kStTimeout);
  }
  __syncthreads();
  return s_go != 0;
}

// ------------------------------------------------------------------ kernels
template <class T>
__global__ void __launch_bounds__(256) k_persistent(KParams<T> kp) {
  __shared__ double red[4][8];
  unsigned gen = 0;
  if (threadIdx.x == 0 && threadIdx.y == 0) gen = ld_acquire_u32(&kp.bar->gen);
  const int nt = *kp.ntiles;
  for (int s = 0; s < kp.nsteps; ++s) {
    for (int t = blockIdx.x; t < nt; t += gridDim.x) pass_a_tile(kp, t, s, red);
    if (!grid_barrier(kp.bar, gen, kp.status, kp.spin_cycles)) return;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) pass_b_tile(kp, t, s);
    if (s + 1 < kp.nsteps && !grid_barrier(kp.bar, gen, kp.status, kp.spin_cycles)) return;
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_pass_a(KParams<T> kp, int s) {
  __shared__ double red[4][8];
  const int nt = *kp.ntiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) pass_a_tile(kp, t, s, red);
}

template <class T>
__global__ void __launch_bounds__(256) k_pass_b(KParams<T> kp, int s) {
  const int nt = *kp.ntiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) pass_b_tile(kp, t, s);
}

// sum(eta) of every tile at the current level (after an initial condition or a restore)
template <class T>
__global__ void __launch_bounds__(256) k_snapshot(KParams<T> kp) {
  __shared__ double red[8];
  const int nt = *kp.ntiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const Tile td = kp.tiles[t];
    const Blk<T> b = RTI_BLK(kp, td.blk);  // copied: see the note on descriptors
    const int p = (int)(kp.scen[b.scen].base & 1);
    double vol = 0.0;
    const int xe = min(td.x0 + kp.tx, b.nx), ye = min(td.y0 + kp.ty, b.ny);
    for (int j = td.y0 + threadIdx.y; j < ye; j += 8)
      for (int i = td.x0 + threadIdx.x; i < xe; i += 32) vol += (double)b.eta[p][ix(b, i, j)];
    vol = warp_sum(vol);
    if (threadIdx.x == 0) red[threadIdx.y] = vol;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      double a = 0.0;
      for (int k = 0; k < 8; ++k) a += red[k];
      b.budget[4 * (size_t)((td.y0 / kp.ty) * b.tiles_x + td.x0 / kp.tx)] = a;
    }
    __syncthreads();
  }
}

// Store the coarse-to-fine edge fluxes of every child block into its current flux
// arrays (parity p), exactly as pass A of the next step will pull them. Used before a
// checkpoint read so that the child's edge faces hold their defined values.
template <class T>
__global__ void __launch_bounds__(256) k_fill_edges(KParams<T> kp, int p) {
  const int nt = *kp.ntiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const Tile td = kp.tiles[t];
    const Blk<T> b = RTI_BLK(kp, td.blk);
    if (!b.is_child) continue;
    const int xe = min(td.x0 + kp.tx, b.nx), ye = min(td.y0 + kp.ty, b.ny);
    for (int j = td.y0 + threadIdx.y; j < ye; j += 8) {
      for (int i = td.x0 + threadIdx.x; i < xe; i += 32) {
        if (i == 0) b.M[p][ix(b, 0, j)] = face_m(kp, b, p, 0, j);
        if (i == b.nx - 1) b.M[p][ix(b, b.nx, j)] = face_m(kp, b, p, b.nx, j);
        if (j == 0) b.N[p][ix(b, i, 0)] = face_n(kp, b, p, i, 0);
        if (j == b.ny - 1) b.N[p][ix(b, i, b.ny)] = face_n(kp, b, p, i, b.ny);
      }
    }
  }
}

// end of a chunk: every scenario advances by the steps it took
__global__ void k_advance(ScenDev* sc, const int* nscen, int nsteps);

}  // namespace rti
