// 2-D / 3-D Crank-Nicolson propagation on sm_103a (tensor-product B-spline basis, Eq. tensor3d).
//
// Per step (Sec. "Time propagation", Eq. cn_system) the system A_n c^{n+1} = B_n c^n with
//   A_n = S + i tau (T + V + sum_a Ebar_a D_a),  B_n = 2S - A_n,
// is solved in correction form c^{n+1} = c^n + delta, A_n delta = r0 = 2 (S c - A_n c), by
// preconditioned COCG (conjugate orthogonal CG for complex symmetric A; bilinear products x^T y).
//
// Operator application (no global matrix is ever formed):
//   * separable terms (S, constant-mass kinetic T, dipoles D_a) are Kronecker products of the
//     per-axis 1-D bands, applied one axis at a time;
//   * the potential V (and, for a position-dependent mass, the kinetic term
//     1/2 sum_a <d_a B| m^-1 |d_a B>, Eq. bdd_elem) by sum factorisation at the Gauss points:
//     interpolate axis by axis to the points, multiply by w_q f(r_q) with f evaluated on the fly
//     from the medium, project back axis by axis (Sec. "Parallel assembly" quadrature).
// In 2-D the non-separable part may instead be assembled once into a (2p+1)^2-point stencil per DoF
// (the same quadrature, summed in advance), which is far cheaper to apply in binary64.
// Preconditioners: the field-free separable operator S(x)S + i tau mbar (T1(x)S + S(x)T1), inverted
// exactly by fast diagonalisation (per-axis generalised eigenvectors T1_a v = lam S_a v; dense
// axis transforms as GEMMs), or the product (x)_a (S_a + i tau mbar T1_a) applied as independent
// banded line solves along each axis.
// Precision: binary64 throughout (TDZ_FP64), or FP32 COCG inside an outer binary64 residual
// refinement (TDZ_MIXED). Reductions accumulate in binary64.
// Observables (Sec. "Dipoles"): norm = c^H S c and d_a = c^H D_a c as Kronecker quadratic forms;
// c^H G_a c (G_a = <m^-1 d_a V>) and c^H K c (K = <m^-1>) as reductions over the Gauss points.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <cstdint>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>
#include <atomic>
#include <thread>

#include "tdz_arith.cuh"
#include "tdz_internal.h"

namespace tdz {
namespace nd {

constexpr int TPB = 256;

struct AxisDev {
  int n, E, nq, Q;
  const double* B;   // [Q][P+1] basis values at point q (element q/nq), column r <-> DoF e + r - 1
  const double* dB;  // [Q][P+1] first derivatives
  const double* x;   // [Q] point coordinates
  const double* w;   // [Q] weights (incl. Jacobian)
  const double* S;   // [n][P+1] lower bands
  const double* T1;
  const double* D;
  // FP32 copies for the single-precision inner solver (no binary64 loads or conversions there)
  const float *fB, *fdB, *fx, *fw, *fS, *fT1, *fD;
  // low parts of B, x, w (value - (double)(float)value): with fB, fx, fw the double-float tables
  const float *lB, *lx, *lw;
  // double-float copies of every table (the binary64-class residual of the mixed path)
  const tdz::fx *xB, *xdB, *xx, *xw, *xS, *xT1, *xD;
  // the absorbing layer's axis factor W_a = <B|eta_a|B> (lower band, as S) in the three precisions, or null
  const double* Wc;
  const float* fWc;
  const tdz::fx* xWc;
};
template <class T> __host__ __device__ inline const T* tab(const AxisDev& A, int which);
template <> __host__ __device__ inline const double* tab<double>(const AxisDev& A, int which) {
  switch (which) { case 0: return A.B; case 1: return A.dB; case 2: return A.x; case 3: return A.w; case 4: return A.S; case 5: return A.T1; case 7: return A.Wc; default: return A.D; }
}
template <> __host__ __device__ inline const tdz::fx* tab<tdz::fx>(const AxisDev& A, int which) {
  switch (which) { case 0: return A.xB; case 1: return A.xdB; case 2: return A.xx; case 3: return A.xw; case 4: return A.xS; case 5: return A.xT1; case 7: return A.xWc; default: return A.xD; }
}
template <> __host__ __device__ inline const float* tab<float>(const AxisDev& A, int which) {
  switch (which) { case 0: return A.fB; case 1: return A.fdB; case 2: return A.fx; case 3: return A.fw; case 4: return A.fS; case 5: return A.fT1; case 7: return A.fWc; default: return A.fD; }
}
enum { TB = 0, TDB = 1, TX = 2, TW = 3, TS = 4, TT1 = 5, TD = 6, TCAP = 7 };

struct MediumDev {
  int mass_kind, pot_kind;
  double mp[4], vp[4];
};

// Medium parameters in the arithmetic type T of a kernel (converted on the host), so that no
// binary64 conversion happens per point in double-float kernels.
template <class T>
struct MediumT {
  int mass_kind, pot_kind;
  T mp[4], vp[4];
  T inv_m0, inv_min, inv_mout;  // 1/mp[0], 1/mp[2], 1/mp[3]
  T w2[3];                      // vp[a]^2 (harmonic oscillator)
};
template <class T>
MediumT<T> medium_t(const MediumDev& d) {
  MediumT<T> m{};
  m.mass_kind = d.mass_kind;
  m.pot_kind = d.pot_kind;
  for (int k = 0; k < 4; ++k) {
    m.mp[k] = (T)d.mp[k];
    m.vp[k] = (T)d.vp[k];
  }
  m.inv_m0 = (T)(1.0 / d.mp[0]);
  m.inv_min = (T)(d.mp[2] != 0.0 ? 1.0 / d.mp[2] : 0.0);
  m.inv_mout = (T)(d.mp[3] != 0.0 ? 1.0 / d.mp[3] : 0.0);
  for (int a = 0; a < 3; ++a) m.w2[a] = (T)(d.vp[a] * d.vp[a]);
  return m;
}

// f(r) at a Gauss point. kind: 0 = V, 1 = 1/2 m^-1 (kinetic weight), 2 = m^-1 dV/dx_axis, 3 = m^-1
template <class T>
__device__ __forceinline__ T medium_f(const MediumT<T>& M, int kind, int axis, const T* r, int dim) {
  T minv = 1;
  if (M.mass_kind == TDZ_MASS_CONST) {
    minv = M.inv_m0;
  } else if (M.mass_kind == TDZ_MASS_ELLIPSE) {
    const T u = r[0] / M.mp[0], v = dim > 1 ? r[1] / M.mp[1] : (T)0;
    minv = (u * u + v * v < (T)1) ? M.inv_min : M.inv_mout;
  }
  if (kind == 1) return (T)0.5f * minv;
  if (kind == 3) return minv;
  T r2 = 0;
  for (int a = 0; a < dim; ++a) r2 += r[a] * r[a];
  if (kind == 0) {
    switch (M.pot_kind) {
      case TDZ_POT_SOFTCORE: return -M.vp[0] / tsqrt(r2 + M.vp[1]);
      case TDZ_POT_HO: {
        T s = 0;
        for (int a = 0; a < dim; ++a) s += M.w2[a] * r[a] * r[a];
        return (T)0.5f * s;
      }
      case TDZ_POT_ELLIPSE: {
        const T u = r[0] / M.vp[0], v = dim > 1 ? r[1] / M.vp[1] : (T)0;
        return (u * u + v * v < (T)1) ? M.vp[2] : M.vp[3];
      }
      default: return 0;
    }
  }
  // kind 2: m^-1 dV/dx_axis
  switch (M.pot_kind) {
    case TDZ_POT_SOFTCORE: {
      const T q = r2 + M.vp[1];
      return minv * M.vp[0] * r[axis] / (q * tsqrt(q));
    }
    case TDZ_POT_HO: return minv * M.w2[axis] * r[axis];
    default: return 0;
  }
}

// reciprocal square root for the FP32 soft-core factor (hardware approximation); the other types never
// take that path
__device__ __forceinline__ float frsqrt(float v) { return rsqrtf(v); }
template <class T>
__device__ __forceinline__ T frsqrt(T v) { return T(1) / tsqrt(v); }

template <class T>
using C = cx<T>;

// Sum-of-products accumulator: a plain multiply-add for float and double; for double-float a
// compensated (Dot2) accumulation, about half the work of double-float multiply-then-add
template <class T>
struct Mac {
  T s;
  TDZ_DEV Mac() : s(0) {}
  TDZ_DEV void add(T a, T b) { s += a * b; }
  TDZ_DEV T get() const { return s; }
};
template <>
struct Mac<fx> {
  ffacc a;
  TDZ_DEV Mac() { acc_zero(a); }
  TDZ_DEV void add(fx x, fx y) { acc_mul(a, to_ff(x), to_ff(y)); }
  TDZ_DEV fx get() const { return to_fx(acc_get(a)); }
};

// ------------------------------------------------------------------------------- axis band terms
// out[o][j][i] (+)= sum_t coef_t * sum_d R_t(j, j+d) in_{sel_t}[o][j+d][i]   (R_t real symmetric bands)
template <class T>
struct BandTerms {
  int nt;
  const void* R[4];
  T cr[4], ci[4];
  int sel[4];
};

// NT = bt.nt terms, interleaved in the neighbour loop: each neighbour value is loaded once per
// input stream and the 2 NT accumulations are independent chains (the double-float Dot2
// accumulations are latency-bound one term at a time)
template <class T, int P, int NT>
__global__ void k_axis_band(BandTerms<T> bt, const C<T>* __restrict__ in0, const C<T>* __restrict__ in1,
                            C<T>* __restrict__ out, long long outer, int L, long long inner, int accumulate) {
  const long long total = outer * L * inner;
  bool need0 = false, need1 = false;  // input streams some term reads
#pragma unroll
  for (int t = 0; t < NT; ++t) (bt.sel[t] ? need1 : need0) = true;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx % inner;
    const long long oj = idx / inner;
    const int j = (int)(oj % L);
    const long long o = oj / L;
    Mac<T> mr[NT], mi[NT];
#pragma unroll
    for (int d = -P; d <= P; ++d) {
      const int jj = j + d;
      if (jj < 0 || jj >= L) continue;
      const size_t bi = (size_t)(jj > j ? jj : j) * (P + 1) + (d < 0 ? -d : d);
      const long long vi = (o * L + jj) * inner + i;
      C<T> v0{}, v1{};
      if (need0) v0 = in0[vi];
      if (need1) v1 = (need0 && in1 == in0) ? v0 : in1[vi];
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const T m = static_cast<const T*>(bt.R[t])[bi];
        const C<T> v = bt.sel[t] ? v1 : v0;
        mr[t].add(m, v.r);
        mi[t].add(m, v.i);
      }
    }
    T ar = 0, ai = 0;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const T sr = mr[t].get(), si = mi[t].get();
      const T cr = bt.cr[t], ci = bt.ci[t];
      ar += cr * sr - ci * si;
      ai += cr * si + ci * sr;
    }
    if (accumulate) {
      C<T> v = out[idx];
      out[idx] = C<T>{v.r + ar, v.i + ai};
    } else {
      out[idx] = C<T>{ar, ai};
    }
  }
}

// one axis pass with bt.nt (1, 3 or 4) terms
template <class T, int P>
void launch_axis_band(cudaStream_t st, int blocks, const BandTerms<T>& bt, const C<T>* in0, const C<T>* in1,
                      C<T>* out, long long outer, int L, long long inner) {
  if (bt.nt == 4)
    k_axis_band<T, P, 4><<<blocks, 256, 0, st>>>(bt, in0, in1, out, outer, L, inner, 0);
  else if (bt.nt == 3)
    k_axis_band<T, P, 3><<<blocks, 256, 0, st>>>(bt, in0, in1, out, outer, L, inner, 0);
  else
    k_axis_band<T, P, 1><<<blocks, 256, 0, st>>>(bt, in0, in1, out, outer, L, inner, 0);
}

// ------------------------------------------------------------------------------- Gauss point passes
// interpolation: out[o][q][i] = sum_r Btab[q][r] in[o][e+r-1][i],  e = q / nq
template <class T, int P>
__global__ void k_interp(const T* __restrict__ Btab, int nq, int n, int Q, const C<T>* __restrict__ in,
                         C<T>* __restrict__ out, long long outer, long long inner) {
  const long long total = outer * Q * inner;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx % inner;
    const long long oq = idx / inner;
    const int q = (int)(oq % Q);
    const long long o = oq / Q;
    const int e = q / nq;
    Mac<T> sr, si;
#pragma unroll
    for (int r = 0; r <= P; ++r) {
      const int j = e + r - 1;
      if (j < 0 || j >= n) continue;
      const T b = Btab[(size_t)q * (P + 1) + r];
      const C<T> v = in[(o * n + j) * inner + i];
      sr.add(b, v.r);
      si.add(b, v.i);
    }
    out[idx] = C<T>{sr.get(), si.get()};
  }
}

// projection: out[o][j][i] = sum_{r, qq} Btab[(e nq + qq)][r] in[o][e nq + qq][i],  e = j + 1 - r
template <class T, int P>
__global__ void k_project(const T* __restrict__ Btab, int nq, int n, int E, const C<T>* __restrict__ in,
                          C<T>* __restrict__ out, long long outer, long long inner, int accumulate) {
  const int Q = E * nq;
  const long long total = outer * n * inner;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx % inner;
    const long long oj = idx / inner;
    const int j = (int)(oj % n);
    const long long o = oj / n;
    Mac<T> mr, mi;
#pragma unroll
    for (int r = 0; r <= P; ++r) {
      const int e = j + 1 - r;
      if (e < 0 || e >= E) continue;
      for (int qq = 0; qq < nq; ++qq) {
        const int q = e * nq + qq;
        const T b = Btab[(size_t)q * (P + 1) + r];
        const C<T> v = in[(o * Q + q) * inner + i];
        mr.add(b, v.r);
        mi.add(b, v.i);
      }
    }
    const T sr = mr.get(), si = mi.get();
    if (accumulate) {
      C<T> v = out[idx];
      out[idx] = C<T>{v.r + sr, v.i + si};
    } else {
      out[idx] = C<T>{sr, si};
    }
  }
}

// The same two passes along an axis whose points have a contiguous inner extent (inner >= 32): one
// thread per (outer, inner) pencil walks the elements with a sliding window of P+1 coefficients, so
// each coefficient (interpolation) or Gauss-point value (projection) is read once and the index
// arithmetic is done once per pencil. The sums are those of k_interp / k_project, the interpolation
// split into even and odd terms.
template <class T, int P>
__global__ void k_interp_win(const T* __restrict__ Btab, int nq, int n, int E, const C<T>* __restrict__ in,
                             C<T>* __restrict__ out, long long outer, long long inner) {
  const long long total = outer * inner;
  const long long Q = (long long)E * nq;
  for (long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x; tid < total;
       tid += (long long)gridDim.x * blockDim.x) {
    const long long i = tid % inner, o = tid / inner;
    const C<T>* src = in + o * n * inner + i;
    C<T>* dst = out + o * Q * inner + i;
    C<T> win[P + 1];  // win[r] = coefficient e + r - 1 of the current element
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      const int j = k - 1;
      win[k] = (j >= 0 && j < n) ? src[(long long)j * inner] : czero<T>();
    }
    for (int e = 0; e < E; ++e) {
      const int jn = e + P;  // enters the window for element e + 1; loaded a whole element ahead
      const C<T> next = (jn < n && e + 1 < E) ? src[(long long)jn * inner] : czero<T>();
      for (int qq = 0; qq < nq; ++qq) {
        const int q = e * nq + qq;
        const T* b = Btab + (size_t)q * (P + 1);
        Mac<T> r0, i0, r1, i1;
#pragma unroll
        for (int k = 0; k <= P; ++k) {
          if (k & 1) {
            r1.add(b[k], win[k].r);
            i1.add(b[k], win[k].i);
          } else {
            r0.add(b[k], win[k].r);
            i0.add(b[k], win[k].i);
          }
        }
        dst[(long long)q * inner] = C<T>{r0.get() + r1.get(), i0.get() + i1.get()};
      }
#pragma unroll
      for (int k = 0; k < P; ++k) win[k] = win[k + 1];
      win[P] = next;
    }
  }
}

template <class T, int P>
__global__ void k_project_win(const T* __restrict__ Btab, int nq, int n, int E, const C<T>* __restrict__ in,
                              C<T>* __restrict__ out, long long outer, long long inner, int accumulate) {
  const long long total = outer * inner;
  const long long Q = (long long)E * nq;
  for (long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x; tid < total;
       tid += (long long)gridDim.x * blockDim.x) {
    const long long i = tid % inner, o = tid / inner;
    const C<T>* src = in + o * Q * inner + i;
    C<T>* dst = out + o * n * inner + i;
    Mac<T> ar[P + 1], ai[P + 1];  // partial projections onto coefficient e + r - 1
    for (int e = 0; e < E; ++e) {
      for (int qq = 0; qq < nq; ++qq) {
        const int q = e * nq + qq;
        const T* b = Btab + (size_t)q * (P + 1);
        const C<T> v = src[(long long)q * inner];
#pragma unroll
        for (int k = 0; k <= P; ++k) {
          ar[k].add(b[k], v.r);
          ai[k].add(b[k], v.i);
        }
      }
      const int j = e - 1;  // coefficient e - 1 is complete
      if (j >= 0 && j < n) {
        C<T>* d = dst + (long long)j * inner;
        const C<T> v = C<T>{ar[0].get(), ai[0].get()};
        if (accumulate) {
          const C<T> u = *d;
          *d = C<T>{u.r + v.r, u.i + v.i};
        } else {
          *d = v;
        }
      }
#pragma unroll
      for (int k = 0; k < P; ++k) {
        ar[k] = ar[k + 1];
        ai[k] = ai[k + 1];
      }
      ar[P] = Mac<T>();
      ai[P] = Mac<T>();
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const int j = E - 1 + k;
      if (j < 0 || j >= n) continue;
      C<T>* d = dst + (long long)j * inner;
      const C<T> v = C<T>{ar[k].get(), ai[k].get()};
      if (accumulate) {
        const C<T> u = *d;
        *d = C<T>{u.r + v.r, u.i + v.i};
      } else {
        *d = v;
      }
    }
  }
}

// The same two passes along the fastest axis (inner = 1): one thread per Gauss point (interpolation) or
// coefficient (projection) of a row, the rows spread over the grid's y dimension, so no index is
// divided per output; the basis values of an interpolation point stay in registers across rows.
template <class T, int P>
__global__ void k_interp_row(const T* __restrict__ Btab, int nq, int n, int Q, const C<T>* __restrict__ in,
                             C<T>* __restrict__ out, long long outer) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const int e = q / nq;
  T bq[P + 1];
#pragma unroll
  for (int r = 0; r <= P; ++r) bq[r] = Btab[(size_t)q * (P + 1) + r];
  for (long long o = blockIdx.y; o < outer; o += gridDim.y) {
    const C<T>* src = in + o * n;
    Mac<T> r0, i0, r1, i1;
#pragma unroll
    for (int r = 0; r <= P; ++r) {
      const int j = e + r - 1;
      if (j < 0 || j >= n) continue;
      const C<T> v = src[j];
      if (r & 1) {
        r1.add(bq[r], v.r);
        i1.add(bq[r], v.i);
      } else {
        r0.add(bq[r], v.r);
        i0.add(bq[r], v.i);
      }
    }
    out[o * Q + q] = C<T>{r0.get() + r1.get(), i0.get() + i1.get()};
  }
}

template <class T, int P>
__global__ void k_project_row(const T* __restrict__ Btab, int nq, int n, int E, const C<T>* __restrict__ in,
                              C<T>* __restrict__ out, long long outer, int accumulate) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const long long Q = (long long)E * nq;
  for (long long o = blockIdx.y; o < outer; o += gridDim.y) {
    const C<T>* src = in + o * Q;
    Mac<T> r0, i0, r1, i1;
#pragma unroll
    for (int r = 0; r <= P; ++r) {
      const int e = j + 1 - r;
      if (e < 0 || e >= E) continue;
      const T* bq = Btab + (size_t)e * nq * (P + 1) + r;
      const C<T>* s = src + (long long)e * nq;
      for (int qq = 0; qq < nq; ++qq) {
        const T bv = bq[(size_t)qq * (P + 1)];
        const C<T> v = s[qq];
        if (qq & 1) {
          r1.add(bv, v.r);
          i1.add(bv, v.i);
        } else {
          r0.add(bv, v.r);
          i0.add(bv, v.i);
        }
      }
    }
    const C<T> v = C<T>{r0.get() + r1.get(), i0.get() + i1.get()};
    C<T>* d = out + o * n + j;
    if (accumulate) {
      const C<T> u = *d;
      *d = C<T>{u.r + v.r, u.i + v.i};
    } else {
      *d = v;
    }
  }
}

template <class T>
struct QGrid {
  int dim;
  int Q[3];
  const T* x[3];
  const T* w[3];
};

// ------------------------------------------------------------------------------- fused last axis
// Along the last (slowest) axis L: for every pencil (one point of the faster axes, already
// interpolated) and chunk of elements, walk the elements with a sliding window of P+1
// coefficients: interpolate to the nq points (table Bl), multiply by coef * w(q) * f(r_q), and
// project back with the same table into out (shape [n_L][inner]; every coefficient is stored once).
// A coefficient completed inside a chunk's element loop is written by that chunk alone; the last
// P partial sums of every chunk but the last (shared with the next chunk) go to `side`
// ([chunk][P][inner]) and k_fused_fixup adds them, so no atomics are needed and the sum order is
// fixed.
template <class T, int P>
__global__ void k_fused_last(const C<T>* __restrict__ in, C<T>* __restrict__ out, C<T>* __restrict__ side,
                             const T* __restrict__ Bl, int nq, int nL, int EL, long long inner, int echunk, QGrid<T> g,
                             MediumT<T> M, int kind, int axis, double cr, double ci, const T* __restrict__ ftab,
                             int stage) {
  const int nchunks = (EL + echunk - 1) / echunk;
  const long long total = inner * nchunks;
  const int L = g.dim - 1;
  const T tcr = (T)cr, tci = (T)ci;
  // with `stage`, the block copies the last axis' basis table (and, without ftab, its point coordinates
  // and weights) to shared memory once: every thread reads the same entries in the same order
  extern __shared__ __align__(16) unsigned char fl_smem[];
  const int QL = EL * nq;
  const T* Bt = Bl;
  const T* xt = g.x[L];
  const T* wt = g.w[L];
  if (stage) {
    T* sB = reinterpret_cast<T*>(fl_smem);
    for (int k = threadIdx.x; k < QL * (P + 1); k += blockDim.x) sB[k] = Bl[k];
    Bt = sB;
    if (!ftab) {
      T* sx = sB + (size_t)QL * (P + 1);
      T* sw = sx + QL;
      for (int k = threadIdx.x; k < QL; k += blockDim.x) {
        sx[k] = g.x[L][k];
        sw[k] = g.w[L][k];
      }
      xt = sx;
      wt = sw;
    }
    __syncthreads();
  }
  // FP32 soft-core potential: f = w (-Z) / sqrt(r^2 + eps) with the pencil's part of r^2 hoisted and a
  // hardware reciprocal square root (the inner solve's precision)
  const bool soft = std::is_same<T, float>::value && kind == 0 && M.pot_kind == TDZ_POT_SOFTCORE;
  for (long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x; tid < total;
       tid += (long long)gridDim.x * blockDim.x) {
    const long long i = tid % inner;
    const int ch = (int)(tid / inner);
    const int e0 = ch * echunk, e1 = min(EL, e0 + echunk);
    // coordinates and weight of the pencil on the faster axes
    T r[3];
    T wp = 1;
    long long t = i;
    for (int a = 0; a < L; ++a) {
      const int q = (int)(t % g.Q[a]);
      t /= g.Q[a];
      r[a] = g.x[a][q];
      wp *= g.w[a][q];
    }
    T r2p = soft ? M.vp[1] : T(0);  // eps + the faster axes' r^2
    if (soft)
      for (int a = 0; a < L; ++a) r2p += r[a] * r[a];
    const T mz = -M.vp[0] * wp;
    C<T> win[P + 1];            // win[r] = coefficient e + r - 1 of the current element
    Mac<T> accr[P + 1], acci[P + 1];  // partial projections onto coefficient e + r - 1
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      const int j = e0 + k - 1;
      win[k] = (j >= 0 && j < nL) ? in[(long long)j * inner + i] : czero<T>();
    }
    // tabulated w(q) f(r_q) of the next kFPre points of the pencil, loaded ahead of use (HBM latency)
    constexpr int kFPre = 4;
    const int qend = e1 * nq;
    T fpre[kFPre];
    if (ftab) {
#pragma unroll
      for (int u = 0; u < kFPre; ++u) {
        const int qp = e0 * nq + u;
        fpre[u] = qp < qend ? ftab[(long long)qp * inner + i] : T(0);
      }
    }
    for (int e = e0; e < e1; ++e) {
      const int jn = e + P;  // coefficient entering the window for element e + 1, loaded a whole element ahead
      const C<T> next = (jn >= 0 && jn < nL && e + 1 < e1) ? in[(long long)jn * inner + i] : czero<T>();
      for (int qq = 0; qq < nq; ++qq) {
        const int q = e * nq + qq;
        const T* b = Bt + (size_t)q * (P + 1);
        // even and odd terms in separate chains (half the dependent latency per point)
        Mac<T> mr0, mi0, mr1, mi1;
#pragma unroll
        for (int k = 0; k <= P; ++k) {
          if (k & 1) {
            mr1.add(b[k], win[k].r);
            mi1.add(b[k], win[k].i);
          } else {
            mr0.add(b[k], win[k].r);
            mi0.add(b[k], win[k].i);
          }
        }
        const T pr = mr0.get() + mr1.get(), pi = mi0.get() + mi1.get();
        T f;
        if (ftab) {  // w(q) f(r_q) tabulated at the Gauss points, [q_L][pencil]
          f = fpre[0];
#pragma unroll
          for (int u = 0; u + 1 < kFPre; ++u) fpre[u] = fpre[u + 1];
          const int qn = q + kFPre;
          fpre[kFPre - 1] = qn < qend ? ftab[(long long)qn * inner + i] : T(0);
        } else if (soft) {
          const T xq = xt[q];
          f = mz * wt[q] * frsqrt(r2p + xq * xq);
        } else {
          r[L] = xt[q];
          f = wp * wt[q] * medium_f<T>(M, kind, axis, r, g.dim);
        }
        const T fr = f * tcr, fi = f * tci;
        const T gr = fr * pr - fi * pi, gi = fr * pi + fi * pr;
#pragma unroll
        for (int k = 0; k <= P; ++k) {
          accr[k].add(b[k], gr);
          acci[k].add(b[k], gi);
        }
      }
      // coefficient e - 1 is complete: emit (its only writer; out needs no clearing); shift both windows
      {
        const int j = e - 1;
        if (j >= 0 && j < nL) out[(long long)j * inner + i] = C<T>{accr[0].get(), acci[0].get()};
      }
#pragma unroll
      for (int k = 0; k < P; ++k) {
        win[k] = win[k + 1];
        accr[k] = accr[k + 1];
        acci[k] = acci[k + 1];
      }
      win[P] = next;
      accr[P] = Mac<T>();
      acci[P] = Mac<T>();
    }
    // remaining partial sums: coefficients e1 - 1 .. e1 + P - 2 (shared with the next chunk)
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const int j = e1 - 1 + k;
      const C<T> a = C<T>{accr[k].get(), acci[k].get()};
      if (e1 < EL) {
        side[((long long)ch * P + k) * inner + i] = a;
      } else if (j >= 0 && j < nL) {
        out[(long long)j * inner + i] = a;
      }
    }
  }
}

// ------------------------------------------------------------------------------- reductions
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// Fixed-order grid reduction, so that repeated runs give bitwise equal sums: every block stores its block
// sums in its own slot of `part`; the last block to arrive (ticket counter) adds the slots in block order -
// the same order whichever block finishes last - and adds the totals to res[0..NV). Called by every thread
// of the block, with v holding the block's sums in thread 0.
struct GridRed {
  double* part;      // [blocks][4]
  unsigned* ticket;  // zero between launches (the last block resets it)
};
template <int NV>
__device__ __forceinline__ void grid_reduce(const double (&v)[NV], double* res, GridRed gr, double* sh) {
  __shared__ int s_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) gr.part[(size_t)blockIdx.x * 4 + k] = v[k];
    __threadfence();
    s_last = atomicAdd(gr.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double t = 0.0;
    for (unsigned q = threadIdx.x; q < gridDim.x; q += blockDim.x) t += __ldcg(gr.part + (size_t)q * 4 + k);
    t = block_sum(t, sh);
    if (threadIdx.x == 0) res[k] += t;
  }
  if (threadIdx.x == 0) *gr.ticket = 0;
}

// k_fused_last for double-float (the mixed path's residual applies): the same pass and the same
// arithmetic, bitwise, with the real and imaginary parts of each complex double-float value carried in
// the two lanes of packed f32x2 registers, so every double-float step serves both parts at once.
__device__ __forceinline__ pcff pcff_load(const C<fx>* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);  // r.h, r.l, i.h, i.l
  return pcff{f2_pack(v.x, v.z), f2_pack(v.y, v.w)};
}
__device__ __forceinline__ void pcff_store(C<fx>* p, pcff a) {
  const float2 h = f2_unpack(a.h), l = f2_unpack(a.l);
  *reinterpret_cast<float4*>(p) = make_float4(h.x, l.x, h.y, l.y);
}
__device__ __forceinline__ pcff pcff_zero() { return pcff{f2_pack(0.f, 0.f), f2_pack(0.f, 0.f)}; }
// (-im, re): multiplication by i
__device__ __forceinline__ pcff pcff_times_i(pcff a) {
  const float2 h = f2_unpack(a.h), l = f2_unpack(a.l);
  return pcff{f2_pack(-h.y, h.x), f2_pack(-l.y, l.x)};
}

// three blocks of 256 per SM (80 registers, some spilled to L1): measured faster than two blocks at 128.
// OBS: the pass also reduces the soft-core observables of its input, whose pencils are those of the
// state c (the first residual apply of a step takes c^n, the state whose observables the previous step
// left open): res[a] += sum_q gtab(q) x_a(q) |psi(q)|^2 for a < dim, i.e. c^H G_a c of Eq.
// pdm_acceleration with gtab = w m^-1 Z (r^2 + eps)^(-3/2) (constant mass). psi(q) is the value the pass
// interpolates for the potential term anyway; along a pencil only x_L varies, so the pencil keeps
// sum_q gtab |psi|^2 and sum_q gtab x_L |psi|^2 and scales the first by the pencil's fixed x_a, a < L.
template <int P, bool OBS>
__global__ void __launch_bounds__(256, 3) k_fused_last_fx(const C<fx>* __restrict__ in, C<fx>* __restrict__ out, C<fx>* __restrict__ side,
                                const fx* __restrict__ Bl, int nq, int nL, int EL, long long inner, int echunk,
                                QGrid<fx> g, MediumT<fx> M, int kind, int axis, double cr, double ci,
                                const fx* __restrict__ ftab, const fx* __restrict__ gtab, double* ores, GridRed gr) {
  const int nchunks = (EL + echunk - 1) / echunk;
  const long long total = inner * nchunks;
  const int L = g.dim - 1;
  const fx tcr = fx(cr), tci = fx(ci);
  const bool imag_only = cr == 0.0;  // the potential term i tau V: no real part to scale
  ffacc oacc[OBS ? 3 : 1];
  if constexpr (OBS)
    for (int a = 0; a < 3; ++a) acc_zero(oacc[a]);
  for (long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x; tid < total;
       tid += (long long)gridDim.x * blockDim.x) {
    const long long i = tid % inner;
    const int ch = (int)(tid / inner);
    const int e0 = ch * echunk, e1 = min(EL, e0 + echunk);
    fx r[3];
    fx wp = 1;
    long long t = i;
    for (int a = 0; a < L; ++a) {
      const int q = (int)(t % g.Q[a]);
      t /= g.Q[a];
      r[a] = g.x[a][q];
      wp *= g.w[a][q];
    }
    ffacc s0, s1;  // OBS: sum gtab |psi|^2 and sum gtab x_L |psi|^2 along this pencil chunk
    acc_zero(s0);
    acc_zero(s1);
    pcff win[P + 1];  // coefficient e + k - 1 of the current element
    pacc acc[P + 1];  // partial projections onto coefficient e + k - 1
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      const int j = e0 + k - 1;
      win[k] = (j >= 0 && j < nL) ? pcff_load(in + (long long)j * inner + i) : pcff_zero();
      pacc_zero(acc[k]);
    }
    constexpr int kFPre = 4;
    const int qend = e1 * nq;
    fx fpre[kFPre];
    if (ftab) {
#pragma unroll
      for (int u = 0; u < kFPre; ++u) {
        const int qp = e0 * nq + u;
        fpre[u] = qp < qend ? ftab[(long long)qp * inner + i] : fx(0);
      }
    }
    for (int e = e0; e < e1; ++e) {
      const int jn = e + P;
      const pcff next = (jn >= 0 && jn < nL && e + 1 < e1) ? pcff_load(in + (long long)jn * inner + i) : pcff_zero();
      for (int qq = 0; qq < nq; ++qq) {
        const int q = e * nq + qq;
        const fx* b = Bl + (size_t)q * (P + 1);
        pacc m0, m1;
        pacc_zero(m0);
        pacc_zero(m1);
#pragma unroll
        for (int k = 0; k <= P; ++k) pacc_mul((k & 1) ? m1 : m0, pfac_of(b[k].h, b[k].l), win[k]);
        const pcff pv = pcff_add(pacc_get(m0), pacc_get(m1));
        if constexpr (OBS) {
          const float2 vh = f2_unpack(pv.h), vl = f2_unpack(pv.l);
          const ff psr = ff{vh.x, vl.x}, psi = ff{vh.y, vl.y};
          ffacc m2;
          acc_zero(m2);
          acc_mul(m2, psr, psr);
          acc_mul(m2, psi, psi);
          const ff wq = ff_mul(acc_get(m2), to_ff(gtab[(long long)q * inner + i]));
          acc_add(s0, wq);
          acc_mul(s1, wq, to_ff(g.x[L][q]));
        }
        fx f;
        if (ftab) {
          f = fpre[0];
#pragma unroll
          for (int u = 0; u + 1 < kFPre; ++u) fpre[u] = fpre[u + 1];
          const int qn = q + kFPre;
          fpre[kFPre - 1] = qn < qend ? ftab[(long long)qn * inner + i] : fx(0);
        } else {
          r[L] = g.x[L][q];
          f = wp * g.w[L][q] * medium_f<fx>(M, kind, axis, r, g.dim);
        }
        const fx fi = f * tci;
        // g = (fr + i fi) p: fr p + fi (i p), lane by lane the scalar fr pr - fi pi, fr pi + fi pr
        pcff gv = pcff_scale(pfac_of(fi.h, fi.l), pcff_times_i(pv));
        if (!imag_only) {
          const fx fr = f * tcr;
          gv = pcff_add(pcff_scale(pfac_of(fr.h, fr.l), pv), gv);
        }
#pragma unroll
        for (int k = 0; k <= P; ++k) pacc_mul(acc[k], pfac_of(b[k].h, b[k].l), gv);
      }
      {
        const int j = e - 1;
        if (j >= 0 && j < nL) pcff_store(out + (long long)j * inner + i, pacc_get(acc[0]));
      }
#pragma unroll
      for (int k = 0; k < P; ++k) {
        win[k] = win[k + 1];
        acc[k] = acc[k + 1];
      }
      win[P] = next;
      pacc_zero(acc[P]);
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const int j = e1 - 1 + k;
      const pcff a = pacc_get(acc[k]);
      if (e1 < EL) {
        pcff_store(side + ((long long)ch * P + k) * inner + i, a);
      } else if (j >= 0 && j < nL) {
        pcff_store(out + (long long)j * inner + i, a);
      }
    }
    if constexpr (OBS) {
      const ff t0 = acc_get(s0);
      for (int a = 0; a < L; ++a) acc_mul(oacc[a], t0, to_ff(r[a]));
      acc_add(oacc[L], acc_get(s1));
    }
  }
  if constexpr (OBS) {
    __shared__ double sh[32];
    double v[3];
    for (int a = 0; a < 3; ++a) {
      const ff t = acc_get(oacc[a]);
      v[a] = block_sum((double)t.h + (double)t.l, sh);
    }
    grid_reduce<3>(v, ores, gr, sh);
  }
}

// w(q) V(r_q) at every Gauss point of a 3-D grid, [q_z][q_y][q_x] (x fastest), evaluated in binary64 and
// stored as double-float: the per-point factor of the potential term of the double-float k_fused_last
// (the FP32 pass evaluates the potential at the points)
__global__ void k_vtab3(AxisDev A0, AxisDev A1, AxisDev A2, MediumT<double> M, fx* __restrict__ tx) {
  const long long total = (long long)A0.Q * A1.Q * A2.Q;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int q0 = (int)(idx % A0.Q);
    const long long t = idx / A0.Q;
    const int q1 = (int)(t % A1.Q), q2 = (int)(t / A1.Q);
    double r[3] = {A0.x[q0], A1.x[q1], A2.x[q2]};
    const double v = A0.w[q0] * A1.w[q1] * A2.w[q2] * medium_f<double>(M, 0, 0, r, 3);
    tx[idx] = fx(v);
  }
}

// w(q) m^-1 Z (r_q^2 + eps)^(-3/2) at every Gauss point of a 2-D/3-D grid (x fastest), in binary64,
// stored as double-float: the point factor of the soft-core observables c^H G_a c (times x_a)
__global__ void k_gtab(AxisDev A0, AxisDev A1, AxisDev A2, int dim, double zm, double eps, fx* __restrict__ tx) {
  const long long total = (long long)A0.Q * A1.Q * (dim > 2 ? A2.Q : 1);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int q0 = (int)(idx % A0.Q);
    const long long t = idx / A0.Q;
    const int q1 = (int)(t % A1.Q), q2 = dim > 2 ? (int)(t / A1.Q) : 0;
    double w = A0.w[q0] * A1.w[q1], r2 = A0.x[q0] * A0.x[q0] + A1.x[q1] * A1.x[q1] + eps;
    if (dim > 2) {
      w *= A2.w[q2];
      r2 += A2.x[q2] * A2.x[q2];
    }
    tx[idx] = fx(w * zm / (r2 * sqrt(r2)));
  }
}

// out[e1(c) - 1 + k] += side[c][k] for every chunk c but the last (after k_fused_last)
template <class T, int P>
__global__ void k_fused_fixup(C<T>* __restrict__ out, const C<T>* __restrict__ side, int nL, long long inner,
                              int echunk, int nchunks) {
  const long long total = (long long)(nchunks - 1) * P * inner;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx % inner;
    const long long t = idx / inner;
    const int k = (int)(t % P);
    const int c = (int)(t / P);
    const int j = (c + 1) * echunk - 1 + k;
    if (j < nL) {
      C<T>* o = out + (long long)j * inner + i;
      const C<T> v = *o, a = side[idx];
      *o = C<T>{v.r + a.r, v.i + a.i};
    }
  }
}

// Medium constants as double-float numbers (prepared on the host once per launch).
struct MediumFF {
  int mass_kind, pot_kind;
  ff m0;                 // 1/m, constant mass
  ff ia, ib, min_, mout; // mass ellipse: 1/a, 1/b, 1/m_in, 1/m_out
  ff z, eps;             // soft core -z / sqrt(r^2 + eps)
  ff w2[3];              // harmonic oscillator w_a^2
};

TDZ_DEV ff ff_sq(ff a) { return ff_mul(a, a); }
// q^(-1/2) for q > 0: FP32 seed refined by one Newton step y + y (1 - q y^2) / 2 with the residual
// in double-float (the seed's ~2^-23 relative error becomes ~2^-46)
TDZ_DEV ff ff_rsqrt(ff q) {
  const float y = rsqrtf(q.h);
  const float p = y * y;
  const ff y2 = ff{p, fmaf(y, y, -p)};
  const ff e = ff_sub(ff{1.0f, 0.0f}, ff_mul(q, y2));
  return ff_add(ff{y, 0.0f}, ff_mulf(e, 0.5f * y));
}

// g[a] = m^-1 dV/dx_a (a < dim) and m^-1 at a Gauss point r, in double-float
TDZ_DEV void medium_grad_ff(const MediumFF& M, const ff* r, int dim, ff* g, ff& minv) {
  minv = M.m0;
  if (M.mass_kind == TDZ_MASS_ELLIPSE) {
    const ff u = ff_mul(r[0], M.ia), v = dim > 1 ? ff_mul(r[1], M.ib) : ff{0.f, 0.f};
    const ff t = ff_add(ff_sq(u), ff_sq(v));
    const bool inside = t.h < 1.0f || (t.h == 1.0f && t.l < 0.0f);
    minv = inside ? M.min_ : M.mout;
  }
  for (int a = 0; a < dim; ++a) g[a] = ff{0.f, 0.f};
  if (M.pot_kind == TDZ_POT_SOFTCORE) {
    ff q = M.eps;
    for (int a = 0; a < dim; ++a) q = ff_add(q, ff_sq(r[a]));
    const ff s = ff_rsqrt(q);
    const ff c = ff_mul(ff_mul(M.z, minv), ff_mul(s, ff_sq(s)));  // z m^-1 q^(-3/2)
    for (int a = 0; a < dim; ++a) g[a] = ff_mul(c, r[a]);
  } else if (M.pot_kind == TDZ_POT_HO) {
    for (int a = 0; a < dim; ++a) g[a] = ff_mul(ff_mul(M.w2[a], r[a]), minv);
  }
}

// Observable reductions at the Gauss points in double-float, fused along the last axis: for every
// pencil (a point of the faster axes, already interpolated) and chunk of elements, psi is
// interpolated to the nq points of each element with a sliding window of P+1 coefficients and
//   res[a] += sum w m^-1 dV/dx_a |psi|^2 (a < dim),  res[3] += sum w m^-1 |psi|^2 (if kmass)
// are accumulated, i.e. c^H G_a c and c^H K c of Eq. pdm_acceleration, without forming the full
// point grid and without binary64 arithmetic per point:
//   res[a] += sum w m^-1 dV/dx_a |psi|^2 (a < dim),  res[3] += sum w m^-1 |psi|^2 (if kmass).
// `in` holds psi interpolated along the faster axes (binary64, shape [nL][inner]).
TDZ_DEV cff to_cff(const C<double>& v) {
  return cff{ff{(float)v.r, (float)(v.r - (double)(float)v.r)}, ff{(float)v.i, (float)(v.i - (double)(float)v.i)}};
}
TDZ_DEV cff to_cff(const C<fx>& v) { return cff{to_ff(v.r), to_ff(v.i)}; }

template <int P, class T>
__global__ void __launch_bounds__(256, 3) k_fused_last_reduce_ff(const C<T>* __restrict__ in, AxisDev A0, AxisDev A1, AxisDev AL, int dim,
                                       long long inner, int echunk, MediumFF M, int kmass,
                                       const fx* __restrict__ gtab, double* res, GridRed gr) {
  __shared__ double sh[32];
  const int nL = AL.n, EL = AL.E, nq = AL.nq;
  const int nchunks = (EL + echunk - 1) / echunk;
  const long long total = inner * nchunks;
  const int L = dim - 1;
  ffacc acc[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) acc_zero(acc[a]);
  for (long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x; tid < total;
       tid += (long long)gridDim.x * blockDim.x) {
    const long long i = tid % inner;
    const int ch = (int)(tid / inner);
    const int e0 = ch * echunk, e1 = min(EL, e0 + echunk);
    ff r[3];
    ff wp = ff{1.f, 0.f};
    {
      long long t = i;
      const AxisDev* F[2] = {&A0, &A1};
      for (int a = 0; a < L; ++a) {
        const AxisDev& A = *F[a];
        const int q = (int)(t % A.Q);
        t /= A.Q;
        r[a] = ff{A.fx[q], A.lx[q]};
        wp = ff_mul(wp, ff{A.fw[q], A.lw[q]});
      }
    }
    ffacc s0, s1;  // tabulated factor: sum gtab |psi|^2 and sum gtab x_L |psi|^2 along this pencil chunk
    acc_zero(s0);
    acc_zero(s1);
    // coefficient e + k - 1 of the current element, real and imaginary parts in the lanes of packed pairs
    auto packed = [](const cff& c) { return pcff{f2_pack(c.r.h, c.i.h), f2_pack(c.r.l, c.i.l)}; };
    pcff win[P + 1];
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      const int j = e0 + k - 1;
      win[k] = packed((j >= 0 && j < nL) ? to_cff(in[(long long)j * inner + i]) : cff{{0.f, 0.f}, {0.f, 0.f}});
    }
    constexpr int kGPre = 4;  // the tabulated factor a few points ahead (the table streams from memory)
    const int gend = e1 * nq;
    fx gpre[kGPre];
    if (gtab) {
#pragma unroll
      for (int u = 0; u < kGPre; ++u) {
        const int qp = e0 * nq + u;
        gpre[u] = qp < gend ? gtab[(long long)qp * inner + i] : fx(0);
      }
    }
    for (int e = e0; e < e1; ++e) {
      // the next element's new coefficient, loaded now so that its latency overlaps this element's points
      const int jn = e + P;
      const cff nxt = (jn >= 0 && jn < nL && e + 1 < e1) ? to_cff(in[(long long)jn * inner + i])
                                                          : cff{{0.f, 0.f}, {0.f, 0.f}};
      for (int qq = 0; qq < nq; ++qq) {
        const int q = e * nq + qq;
        const float* bh = AL.fB + (size_t)q * (P + 1);
        const float* bl = AL.lB + (size_t)q * (P + 1);
        pacc pm;  // the state at the point (both parts in one Dot2 chain of packed pairs)
        pacc_zero(pm);
#pragma unroll
        for (int k = 0; k <= P; ++k) pacc_mul(pm, pfac_of(bh[k], bl[k]), win[k]);
        const pcff pv = pacc_get(pm);
        const float2 vh = f2_unpack(pv.h), vl = f2_unpack(pv.l);
        const ff psr = ff{vh.x, vl.x}, psi = ff{vh.y, vl.y};
        ffacc m2;
        acc_zero(m2);
        acc_mul(m2, psr, psr);
        acc_mul(m2, psi, psi);
        r[L] = ff{AL.fx[q], AL.lx[q]};
        if (gtab) {  // w m^-1 Z (r^2 + eps)^(-3/2) tabulated: the soft-core gradient is that times r_a
          const ff wq = ff_mul(acc_get(m2), to_ff(gpre[0]));
#pragma unroll
          for (int u = 0; u + 1 < kGPre; ++u) gpre[u] = gpre[u + 1];
          gpre[kGPre - 1] = q + kGPre < gend ? gtab[(long long)(q + kGPre) * inner + i] : fx(0);
          acc_add(s0, wq);        // r_a, a < L, is fixed along the pencil: applied once, below
          acc_mul(s1, wq, r[L]);
        } else {
          const ff wq = ff_mul(ff_mul(wp, ff{AL.fw[q], AL.lw[q]}), acc_get(m2));
          ff g[3], minv;
          medium_grad_ff(M, r, dim, g, minv);
          for (int a = 0; a < dim; ++a) acc_mul(acc[a], wq, g[a]);
          if (kmass) acc_mul(acc[3], wq, minv);
        }
      }
#pragma unroll
      for (int k = 0; k < P; ++k) win[k] = win[k + 1];
      win[P] = packed(nxt);
    }
    if (gtab) {
      const ff t0 = acc_get(s0);
      for (int a = 0; a < L; ++a) acc_mul(acc[a], t0, r[a]);
      acc_add(acc[L], acc_get(s1));
    }
  }
  double v[4];
  for (int a = 0; a < 4; ++a) {
    const ff t = acc_get(acc[a]);
    v[a] = block_sum((double)t.h + (double)t.l, sh);
  }
  grid_reduce<4>(v, res, gr, sh);
}

// res[0] += Re sum conj(a) b ; res[1] += Im   (Hermitian product, for observables)
template <class T>
__global__ void k_hdot(const C<T>* __restrict__ a, const C<T>* __restrict__ b, long long n, double* res,
                       GridRed gr) {
  __shared__ double sh[32];
  double re = 0.0, im = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C<T> x = a[i], y = b[i];
    re += (double)x.r * (double)y.r + (double)x.i * (double)y.i;
    im += (double)x.r * (double)y.i - (double)x.i * (double)y.r;
  }
  re = block_sum(re, sh);
  im = block_sum(im, sh);
  const double sums[2] = {re, im};
  grid_reduce<2>(sums, res, gr, sh);
}

// res[0..1] += sum a b (bilinear, no conjugation: COCG); res[2] += ||b||^2 if nrm
template <class T>
__global__ void k_bdot(const C<T>* __restrict__ a, const C<T>* __restrict__ b, long long n, double* res,
                       GridRed gr) {
  __shared__ double sh[32];
  double re = 0.0, im = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C<T> x = a[i], y = b[i];
    re += (double)x.r * (double)y.r - (double)x.i * (double)y.i;
    im += (double)x.r * (double)y.i + (double)x.i * (double)y.r;
  }
  re = block_sum(re, sh);
  im = block_sum(im, sh);
  const double sums[2] = {re, im};
  grid_reduce<2>(sums, res, gr, sh);
}

// The Kronecker quadratic forms of the 2-D observables in one pass along y, given t = S_x c and
// u = D_x c (x-passes): res[0] += c^H (S_y(x)S_x) c (norm), res[1] += c^H (S_y(x)D_x) c (d_x),
// res[2] += c^H (D_y(x)S_x) c (d_y); the y-sums in the arithmetic T, the products with conj(c) and the
// accumulation in binary64 (real parts: the forms are Hermitian)
template <class T, int P>
__global__ void k_qform2_y(const C<T>* __restrict__ c, const C<T>* __restrict__ t, const C<T>* __restrict__ u,
                           const T* __restrict__ Sy, const T* __restrict__ Dy, int nx, int ny, double* res,
                           GridRed gr) {
  __shared__ double sh[32];
  double q0 = 0.0, q1 = 0.0, q2 = 0.0;
  const long long N = (long long)nx * ny;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(idx % nx), iy = (int)(idx / nx);
    Mac<T> sr, si, dr, di, ur, ui;
#pragma unroll
    for (int d = -P; d <= P; ++d) {
      const int jy = iy + d;
      if (jy < 0 || jy >= ny) continue;
      const size_t bi = (size_t)(jy > iy ? jy : iy) * (P + 1) + (d < 0 ? -d : d);
      const T sv = Sy[bi], dv = Dy[bi];
      const C<T> tv = t[(long long)jy * nx + ix], uv = u[(long long)jy * nx + ix];
      sr.add(sv, tv.r);
      si.add(sv, tv.i);
      dr.add(dv, tv.r);
      di.add(dv, tv.i);
      ur.add(sv, uv.r);
      ui.add(sv, uv.i);
    }
    const C<T> cv = c[idx];
    const double cr = (double)cv.r, ci = (double)cv.i;
    q0 += cr * (double)sr.get() + ci * (double)si.get();
    q1 += cr * (double)ur.get() + ci * (double)ui.get();
    q2 += cr * (double)dr.get() + ci * (double)di.get();
  }
  q0 = block_sum(q0, sh);
  q1 = block_sum(q1, sh);
  q2 = block_sum(q2, sh);
  const double v[3] = {q0, q1, q2};
  grid_reduce<3>(v, res, gr, sh);
}



// a / b for complex binary64 scalars, 0 when b = 0
__device__ __forceinline__ double2 cdiv_or_zero(const double* a, const double* b) {
  const double br = b[0], bi = b[1];
  const double d = br * br + bi * bi;
  if (d == 0.0) return make_double2(0.0, 0.0);
  return make_double2((a[0] * br + a[1] * bi) / d, (a[1] * br - a[0] * bi) / d);
}

// COCG update: x += alpha p; r -= alpha q; res[0] += ||r||^2, with alpha = rho / (p^T q) read from the
// reduction slots (0 when p^T q = 0)
template <class T>
__global__ void k_cocg_update_dev(C<T>* __restrict__ x, C<T>* __restrict__ r, const C<T>* __restrict__ p,
                                  const C<T>* __restrict__ q, long long n, const double* rho, const double* pq,
                                  double* res, GridRed gr) {
  __shared__ double sh[32];
  __shared__ double2 s_al;  // one complex division per block, not per thread (the FP64 rate is low)
  if (threadIdx.x == 0) s_al = cdiv_or_zero(rho, pq);
  __syncthreads();
  const double2 al = s_al;
  double acc = 0.0;
  const T a_r = (T)al.x, a_i = (T)al.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C<T> pv = p[i], qv = q[i];
    C<T> xv = x[i], rv = r[i];
    xv.r += a_r * pv.r - a_i * pv.i;
    xv.i += a_r * pv.i + a_i * pv.r;
    rv.r -= a_r * qv.r - a_i * qv.i;
    rv.i -= a_r * qv.i + a_i * qv.r;
    x[i] = xv;
    r[i] = rv;
    acc += (double)rv.r * (double)rv.r + (double)rv.i * (double)rv.i;
  }
  acc = block_sum(acc, sh);
  const double v[1] = {acc};
  grid_reduce<1>(v, res, gr, sh);
}

// p = z + beta p with beta = rho_new / rho read from the reduction slots (0 when rho = 0)
template <class T>
__global__ void k_xpby_dev(C<T>* __restrict__ p, const C<T>* __restrict__ z, long long n, const double* rho_new,
                           const double* rho) {
  __shared__ double2 s_be;  // one complex division per block
  if (threadIdx.x == 0) s_be = cdiv_or_zero(rho_new, rho);
  __syncthreads();
  const double2 be = s_be;
  const T b_r = (T)be.x, b_i = (T)be.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C<T> pv = p[i], zv = z[i];
    p[i] = C<T>{zv.r + b_r * pv.r - b_i * pv.i, zv.i + b_r * pv.i + b_i * pv.r};
  }
}

// y = a*x + b*y  (real scalars), mixed types (Tx -> Ty)
template <class Tx, class Ty>
__global__ void k_axby(const C<Tx>* __restrict__ x, C<Ty>* __restrict__ y, long long n, double a, double b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C<Tx> xv = x[i];
    if (b == 0.0) {  // y is output only
      y[i] = C<Ty>{(Ty)(a * (double)xv.r), (Ty)(a * (double)xv.i)};
      continue;
    }
    const C<Ty> yv = y[i];
    y[i] = C<Ty>{(Ty)(a * (double)xv.r + b * (double)yv.r), (Ty)(a * (double)xv.i + b * (double)yv.i)};
  }
}

// y = (ar + i ai) x + (br + i bi) y; x may alias y (each element is read and written by one thread)
template <class T>
__global__ void k_caxpby(const C<T>* x, C<T>* y, long long n, double ar, double ai, double br, double bi) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C<T> u = x[i], v = y[i];
    const T xr = u.r, xi = u.i, yr = v.r, yi = v.i;
    y[i] = C<T>{(T)(ar * xr - ai * xi + br * yr - bi * yi), (T)(ar * xi + ai * xr + br * yi + bi * yr)};
  }
}

template <class T>
__global__ void k_nrm(const C<T>* __restrict__ a, long long n, double* res, GridRed gr) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const C<T> x = a[i];
    acc += (double)x.r * (double)x.r + (double)x.i * (double)x.i;
  }
  acc = block_sum(acc, sh);
  const double v[1] = {acc};
  grid_reduce<1>(v, res, gr, sh);
}

// ------------------------------------------------------------------------------- preconditioner
// per line along an axis: solve P u = v in place, P = L D L^T with Lc[j][d-1] = L(j+d, j), Dv = D^-1
template <class T, int P>
__global__ void k_line_solve(C<T>* __restrict__ v, const C<T>* __restrict__ Lc, const C<T>* __restrict__ Dv,
                             long long outer, int n, long long inner) {
  const long long lines = outer * inner;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < lines;
       l += (long long)gridDim.x * blockDim.x) {
    const long long i = l % inner, o = l / inner;
    C<T>* base = v + o * n * inner + i;
    C<T> win[P + 1];
#pragma unroll
    for (int d = 0; d <= P; ++d) win[d] = czero<T>();
    for (int j = 0; j < n; ++j) {  // forward: y_j = v_j - sum_d L(j, j-d) y_{j-d}
      C<T> y = base[(long long)j * inner];
#pragma unroll
      for (int d = 1; d <= P; ++d)
        if (j - d >= 0) y = cmsub(y, Lc[(size_t)(j - d) * P + d - 1], win[d]);
#pragma unroll
      for (int d = P; d >= 2; --d) win[d] = win[d - 1];
      win[1] = y;
      base[(long long)j * inner] = cmul(y, Dv[j]);
    }
#pragma unroll
    for (int d = 0; d <= P; ++d) win[d] = czero<T>();
    for (int j = n - 1; j >= 0; --j) {  // backward: x_j = z_j - sum_d L(j+d, j) x_{j+d}
      C<T> x = base[(long long)j * inner];
#pragma unroll
      for (int d = 1; d <= P; ++d)
        if (j + d < n) x = cmsub(x, Lc[(size_t)j * P + d - 1], win[d]);
#pragma unroll
      for (int d = P; d >= 2; --d) win[d] = win[d - 1];
      win[1] = x;
      base[(long long)j * inner] = x;
    }
  }
}

// ------------------------------------------------------------------------------- 2-D stencil operator
// FP32 stencil tiles: kWtRows consecutive x-indices of one grid row iy (a tile never crosses a grid
// row; the last tile of a row is zero padded), layout [tile][offset][row in tile] with tile index
// iy * ceil(nx / kWtRows) + ix / kWtRows
constexpr int kWtRows = 64;  // rows per stencil tile

__host__ __device__ inline int wt_tiles_per_row(int nx) { return (nx + kWtRows - 1) / kWtRows; }
__host__ __device__ inline size_t wt_index(int noff, int off, int ix, int iy, int nx) {
  const size_t tile = (size_t)iy * wt_tiles_per_row(nx) + ix / kWtRows;
  return (tile * noff + off) * kWtRows + (size_t)(ix % kWtRows);
}

// In 2-D the non-separable part of H (the potential and, for a position-dependent mass, the kinetic
// term 1/2 <d_a B| m^-1 |d_a B>, Sec. "Parallel assembly") couples DoF (ix, iy) only with
// (ix + dx, iy + dy), |dx|, |dy| <= P. It is assembled once, exactly as the Gauss-point quadrature
// defines it, by sum factorisation:
//   table:   fV(x_qx, y_qy) = V, fK = 1/2 m^-1 at every Gauss point
//   stage 1: F1[qy][dx][ix] = sum_{qx} w_x (fV B_ix B_jx + fK dB_ix dB_jx),
//            F2[qy][dx][ix] = sum_{qx} w_x  fK B_ix B_jx                   (variable mass only)
//   stage 2: W[(dy, dx)][iy nx + ix] = sum_{qy} w_y (B_iy B_jy F1 + dB_iy dB_jy F2),
// with jx = ix + dx, jy = iy + dy. Binary64 and double-float copies: symmetric half, layout
// [offset][row], so that a warp reads one offset of 32 consecutive rows in one transaction. FP32
// copy: the full stencil, tile-major (see the fused 2-D apply).
__global__ void k_w_ftab(AxisDev ax, AxisDev ay, MediumT<double> M, int varmass, double* __restrict__ fV,
                         double* __restrict__ fK) {
  const long long total = (long long)ax.Q * ay.Q;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    double r[2];
    r[0] = ax.x[idx % ax.Q];
    r[1] = ay.x[idx / ax.Q];
    fV[idx] = medium_f<double>(M, 0, 0, r, 2);
    if (varmass) fK[idx] = medium_f<double>(M, 1, 0, r, 2);
  }
}

// one thread per (qy, ix): the 2P+1 offsets dx from the elements of ix (local index ri) and their
// functions jx = e + rj - 1
template <int P>
__global__ void k_w_stage1(AxisDev ax, AxisDev ay, int varmass, const double* __restrict__ fV,
                           const double* __restrict__ fK, double* __restrict__ F1, double* __restrict__ F2) {
  constexpr int W = 2 * P + 1;
  const long long total = (long long)ay.Q * ax.n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(idx % ax.n);
    const int qy = (int)(idx / ax.n);
    double s1[W], s2[W];
#pragma unroll
    for (int t = 0; t < W; ++t) s1[t] = s2[t] = 0.0;
    const int e0 = max(0, ix + 1 - P), e1 = min(ax.E - 1, ix + 1);
    for (int e = e0; e <= e1; ++e) {
      const int ri = ix + 1 - e;
      for (int qq = 0; qq < ax.nq; ++qq) {
        const int q = e * ax.nq + qq;
        const double* Bq = ax.B + (size_t)q * (P + 1);
        const double* dBq = ax.dB + (size_t)q * (P + 1);
        const double wv = ax.w[q] * fV[(size_t)qy * ax.Q + q];
        const double wk = varmass ? ax.w[q] * fK[(size_t)qy * ax.Q + q] : 0.0;
        const double bi = Bq[ri], dbi = dBq[ri];
#pragma unroll
        for (int rj = 0; rj <= P; ++rj) {
          const int dxi = e + rj - 1 - ix + P;  // in [0, 2P] since both functions live on element e
          const double bb = bi * Bq[rj];
          s1[dxi] += wv * bb + (varmass ? wk * dbi * dBq[rj] : 0.0);
          if (varmass) s2[dxi] += wk * bb;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < W; ++t) {
      const int jx = ix + t - P;
      const bool in = jx >= 0 && jx < ax.n;  // Dirichlet-trimmed functions do not couple
      const size_t o = ((size_t)qy * W + t) * ax.n + ix;
      F1[o] = in ? s1[t] : 0.0;
      if (varmass) F2[o] = in ? s2[t] : 0.0;
    }
  }
}

// W is symmetric (W_{i,j} = W_{j,i}), so only the offsets (dy, dx) with dy > 0, or dy = 0 and dx >= 0,
// are stored: (P+1) + P(2P+1) of them, W_{(ix,iy),(ix+dx,iy+dy)} at [half_off(dy, dx)][iy nx + ix]
__host__ __device__ constexpr int half_count(int P) { return (P + 1) + P * (2 * P + 1); }
__host__ __device__ constexpr int half_off(int P, int dy, int dx) {
  return dy == 0 ? dx : (P + 1) + (dy - 1) * (2 * P + 1) + (dx + P);
}

// one thread per (iy, dx, ix): the 2P+1 offsets dy (the stored half of them)
template <int P>
__global__ void k_w_stage2(AxisDev ax, AxisDev ay, int varmass, const double* __restrict__ F1,
                           const double* __restrict__ F2, double* __restrict__ W64, float* __restrict__ W32,
                           fx* __restrict__ Wx) {
  constexpr int W = 2 * P + 1;
  const long long N = (long long)ax.n * ay.n;
  const long long total = N * W;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(idx % ax.n);
    const long long t = idx / ax.n;
    const int dxi = (int)(t % W);
    const int iy = (int)(t / W);
    double s[W];
#pragma unroll
    for (int k = 0; k < W; ++k) s[k] = 0.0;
    const int e0 = max(0, iy + 1 - P), e1 = min(ay.E - 1, iy + 1);
    for (int e = e0; e <= e1; ++e) {
      const int ri = iy + 1 - e;
      for (int qq = 0; qq < ay.nq; ++qq) {
        const int q = e * ay.nq + qq;
        const double* Bq = ay.B + (size_t)q * (P + 1);
        const double* dBq = ay.dB + (size_t)q * (P + 1);
        const size_t f = ((size_t)q * W + dxi) * ax.n + ix;
        const double a1 = ay.w[q] * Bq[ri] * F1[f];
        const double a2 = varmass ? ay.w[q] * dBq[ri] * F2[f] : 0.0;
#pragma unroll
        for (int rj = 0; rj <= P; ++rj) {
          const int dyi = e + rj - 1 - iy + P;
          s[dyi] += a1 * Bq[rj] + (varmass ? a2 * dBq[rj] : 0.0);
        }
      }
    }
    const long long row = (long long)iy * ax.n + ix;
    const int dx = dxi - P;
    const int jx = ix + dx;
#pragma unroll
    for (int dyi = 0; dyi < W; ++dyi) {
      const int dy = dyi - P;
      const int jy = iy + dy;
      const bool in = jx >= 0 && jx < ax.n && jy >= 0 && jy < ay.n;
      const double v = in ? s[dyi] : 0.0;
      if (W32) W32[wt_index(W * W, dyi * W + dxi, ix, iy, ax.n)] = (float)v;  // full stencil, tile-major
      if (dy < 0 || (dy == 0 && dx < 0)) continue;
      const size_t o = (size_t)half_off(P, dy, dx) * N + row;  // half layout
      if (W64) W64[o] = v;
      if (Wx) Wx[o] = fx(v);
    }
  }
}

// y += i tau W x  (W real symmetric; stored half, see half_off): each stored entry serves row i with
// neighbour i + off and, transposed, row i with neighbour i - off (read at row i - off: coalesced)
template <class T, int P>
__global__ void k_wapply(const T* __restrict__ Wm, const C<T>* __restrict__ x, C<T>* __restrict__ y, int nx, int ny,
                         T tau) {
  const long long N = (long long)nx * ny;
  for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < N;
       row += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(row % nx), iy = (int)(row / nx);
    Mac<T> mr, mi;
#pragma unroll 1
    for (int dy = 0; dy <= P; ++dy) {
      const T* wr = Wm + (size_t)half_off(P, dy, 0) * N;
#pragma unroll
      for (int dx = -P; dx <= P; ++dx) {
        if (dy == 0 && dx < 0) continue;
        const T* wo = wr + (long long)dx * N;  // offset (dy, dx) is stored at half_off(P, dy, 0) + dx
        const int jx = ix + dx, jy = iy + dy;
        if (jx >= 0 && jx < nx && jy < ny) {  // direct: W_{row, row + (dx, dy)}
          const T w = wo[row];
          const C<T> v = x[(long long)jy * nx + jx];
          mr.add(w, v.r);
          mi.add(w, v.i);
        }
        const int kx = ix - dx, ky = iy - dy;
        if ((dy > 0 || dx > 0) && kx >= 0 && kx < nx && ky >= 0) {  // transposed: W_{row - off, row}
          const long long rr = (long long)ky * nx + kx;
          const T w = wo[rr];
          const C<T> v = x[rr];
          mr.add(w, v.r);
          mi.add(w, v.i);
        }
      }
    }
    const T sr = mr.get(), si = mi.get();
    const C<T> o = y[row];
    y[row] = C<T>{o.r - tau * si, o.i + tau * sr};
  }
}

// ------------------------------------------------------------------ fused 2-D apply (FP32 inner solve)
// y = A_n x for a 2-D tensor basis in one pass over memory:
//   A_n = S_y(x)(S_x + i tau K_x) + i tau K_y(x)S_x + i tau W,   K_a = cm T1_a + Ebar_a D_a,
// i.e. the Kronecker terms of the separable operator (evaluated on the fly from per-axis coefficient
// rows) plus the assembled non-separable stencil W. W is the only large operand (4 (2P+1)^2 bytes per
// DoF); it is stored tile-major (tiles of kWtRows x-indices of one grid row), so that a tile is one
// contiguous block that a single bulk TMA copy moves into shared memory. A persistent CTA streams
// its tiles through a ring of stages (mbarrier completion, every wait bounded) with the copies of the
// next tiles in flight, and stages the (2P+1) x (kWtRows + 2P) neighbourhood of x one tile ahead.

// per-axis coefficient rows of the separable part: out[i][k] = {S(i, j), cm T1(i, j) + e D(i, j)},
// j = i + k - P, k = 0..2P; zero where j is outside [0, n) and in the pad entry k = 2P + 1
template <int P>
__global__ void k_rowband(const float* __restrict__ S, const float* __restrict__ T1, const float* __restrict__ D,
                          int n, float cm, float e, float2* __restrict__ out) {
  constexpr int PW = 2 * P + 2;
  const long long total = (long long)n * PW;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / PW), k = (int)(idx % PW);
    const int d = k - P, j = i + d;
    float2 v = make_float2(0.f, 0.f);
    if (k <= 2 * P && j >= 0 && j < n) {
      const size_t o = (size_t)(j > i ? j : i) * (P + 1) + (d < 0 ? -d : d);
      v = make_float2(S[o], cm * T1[o] + e * D[o]);
    }
    out[idx] = v;
  }
}

// ---- bulk-copy / mbarrier primitives (inline PTX, sm_90+ forms available on sm_103a)
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// contiguous global -> shared copy by the TMA unit; completion is signalled on the mbarrier
// (addresses 16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the phase with the given parity to complete; gives up after `limit` SM cycles
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
constexpr long long kWaitLimit = 4000000000LL;    // about 2 s at the maximum SM clock
constexpr long long kWaitLimitTest = 20000000LL;  // about 10 ms (TDZ_OPT_WAIT_TEST)

template <int P, int G>
struct Apply2dCfg {
  static constexpr int W = 2 * P + 1;
  static constexpr int NOFF = W * W;
  static constexpr int R = kWtRows;
  static constexpr int HW = R + 2 * P;                 // halo width (x-indices) of a tile
  static constexpr int PW = 2 * P + 2;                 // coefficient row length (float2)
  static constexpr int XH = W * HW;                    // float2: (2P+1) rows of x around the tile
  static constexpr int CB = R * PW;                    // float2: coefficient rows of the tile's x-indices
  // per tile, one buffer: x halo, then the x-axis coefficient rows as [j][row parity][row / 2] float4
  // (conflict-free when lane l reads rows 2l and 2l + 1), then the y-axis coefficient row of iy
  static constexpr int HALO_BYTES = (XH + CB + PW) * 8;
  static constexpr int STAGE_BYTES = NOFF * R * 4;
  static constexpr int RED_BYTES = 2 * (G - 1) * R * 8;
  static constexpr int FIXED = RED_BYTES + 2 * HALO_BYTES + 64;
  static constexpr int NST = (3 * STAGE_BYTES + FIXED <= 227 * 1024) ? 3 : 2;
  static constexpr int THREADS = 32 * G;               // one warp per group; a lane owns two rows
  static constexpr size_t SMEM = (size_t)NST * STAGE_BYTES + RED_BYTES + 2 * HALO_BYTES + 8 * NST;
};

// cp.async of one float2 into shared memory, zero-filled when `in` is false (nothing is read then)
__device__ __forceinline__ void cp_async8(uint32_t dst, const float2* src, bool in) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(in ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool in) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// packed FP32 pair: d = a * b + c on both lanes (one f32x2 instruction)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }

// Everything a tile (iy, bx) reads besides its stencil block, into one shared buffer h:
//   h[(dy + P) * HW + c] = x(iy + dy, bx * R - P + c)   (zero outside the grid),
//   x-axis coefficient rows of ix = bx * R + row (zero beyond nx) at XH as float4 [j][row & 1][row / 2],
//   the y-axis coefficient row of iy at XH + CB.
template <int P, int G>
__device__ __forceinline__ void load_halo(float2* h, const float2* __restrict__ x, const float2* __restrict__ xb,
                                          const float2* __restrict__ yb, int iy, int bx, int nx, int ny) {
  using Cfg = Apply2dCfg<P, G>;
  constexpr int HW = Cfg::HW, HE = Cfg::XH, R = Cfg::R, PW = Cfg::PW, NJ = PW / 2;
  const int jx0 = bx * R - P;
  for (int e = threadIdx.x; e < HE; e += Cfg::THREADS) {
    const int jy = iy + e / HW - P, jx = jx0 + e % HW;
    const bool in = jy >= 0 && jy < ny && jx >= 0 && jx < nx;
    cp_async8(smem_addr(h + e), in ? x + (long long)jy * nx + jx : x, in);
  }
  float4* cb = reinterpret_cast<float4*>(h + HE);
  for (int e = threadIdx.x; e < R * NJ; e += Cfg::THREADS) {
    const int row = e / NJ, j = e % NJ, ix = bx * R + row;
    const bool in = ix < nx;
    cp_async16(smem_addr(cb + (j * 2 + (row & 1)) * (R / 2) + row / 2), in ? xb + (size_t)ix * PW + 2 * j : xb, in);
  }
  for (int e = threadIdx.x; e < NJ; e += Cfg::THREADS)
    cp_async16(smem_addr(reinterpret_cast<float4*>(h + HE + Cfg::CB) + e), yb + (size_t)iy * PW + 2 * e, true);
  cp_async_commit();
}

// Offsets dy0 .. dy0 + PER - 1 of the two rows rl, rl + 1 of a lane (h: halo at column rl, w: stage
// at row rl). Per row and dy: a_S += S_y u_S and a_T += S_y u_K + K_y u_S + u_W, with u_S, u_K, u_W
// the sums over dx of S_x x, K_x x and W x along grid row jy = iy + dy of x (zero outside the grid,
// so no bounds checks). The 2P+2 halo values of both rows come as float4 loads, W of both rows as
// one float2 per offset; complex-times-real products are packed f32x2 FMAs.
template <int P, int G, int PER>
__device__ __forceinline__ void stencil_pair(const float2* h, const float* w, const float2* cyv,
                                             const float2 (&b0)[2 * P + 2], const float2 (&b1)[2 * P + 2], int dy0,
                                             float2 (&aS)[2], float2 (&aT)[2]) {
  using Cfg = Apply2dCfg<P, G>;
  constexpr int W = 2 * P + 1, R = kWtRows, HW = Cfg::HW, PW = 2 * P + 2;
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int dy = dy0 + t;
    if (dy > P) break;
    const float2 cy = cyv[t];
    const float4* xr4 = reinterpret_cast<const float4*>(h + (dy + P) * HW);
    float2 xv[PW];
#pragma unroll
    for (int j = 0; j < PW / 2; ++j) {
      const float4 v = xr4[j];
      xv[2 * j] = make_float2(v.x, v.y);
      xv[2 * j + 1] = make_float2(v.z, v.w);
    }
    const float2* wr = reinterpret_cast<const float2*>(w + (dy + P) * W * R);
    float2 uS0 = splat(0.f), uK0 = splat(0.f), uW0 = splat(0.f), uS1 = splat(0.f), uK1 = splat(0.f),
           uW1 = splat(0.f);
#pragma unroll
    for (int d = 0; d < W; ++d) {
      const float2 wd = wr[d * (R / 2)];  // {W(row rl), W(row rl + 1)} at offset d
      uS0 = ffma2(splat(b0[d].x), xv[d], uS0);
      uK0 = ffma2(splat(b0[d].y), xv[d], uK0);
      uW0 = ffma2(splat(wd.x), xv[d], uW0);
      uS1 = ffma2(splat(b1[d].x), xv[d + 1], uS1);
      uK1 = ffma2(splat(b1[d].y), xv[d + 1], uK1);
      uW1 = ffma2(splat(wd.y), xv[d + 1], uW1);
    }
    aS[0] = ffma2(splat(cy.x), uS0, aS[0]);
    aS[1] = ffma2(splat(cy.x), uS1, aS[1]);
    aT[0] = ffma2(splat(cy.x), uK0, ffma2(splat(cy.y), uS0, make_float2(aT[0].x + uW0.x, aT[0].y + uW0.y)));
    aT[1] = ffma2(splat(cy.x), uK1, ffma2(splat(cy.y), uS1, make_float2(aT[1].x + uW1.x, aT[1].y + uW1.y)));
  }
}

// One warp per group g of offsets dy; lane l owns rows rl = 2l, 2l + 1 of the tile. Group 0 adds
// up the G partial sums (double-buffered in shared memory by tile parity, so one barrier per tile
// suffices). Per tile: the stencil block arrives by bulk copy (ring of NST stages, issued NST tiles
// ahead), the x halo by zero-filling cp.async (one tile ahead). err: set to 1 if a stencil copy did
// not complete in time. wait_limit: SM cycles a wait may take; issue = 0 (test aid) issues no
// stencil copies, so that the first wait runs out and the error path is taken.
template <int P, int G>
__global__ void __launch_bounds__(32 * G, 1)
    k_apply2d_tma(const float* __restrict__ Wt, long long ntiles, const float2* __restrict__ x, float2* __restrict__ y,
                  const float2* __restrict__ xb, const float2* __restrict__ yb, int nx, int ny, float tau,
                  int* __restrict__ err, long long wait_limit, int issue) {
  using Cfg = Apply2dCfg<P, G>;
  constexpr int R = Cfg::R, NST = Cfg::NST, PW = 2 * P + 2;
  constexpr int PER = (2 * P + 1 + G - 1) / G;  // offsets dy per group
  extern __shared__ __align__(128) unsigned char smem[];
  float* stages = reinterpret_cast<float*>(smem);
  float2* red = reinterpret_cast<float2*>(smem + (size_t)NST * Cfg::STAGE_BYTES);
  float2* halo = reinterpret_cast<float2*>(smem + (size_t)NST * Cfg::STAGE_BYTES + Cfg::RED_BYTES);
  uint64_t* bars =
      reinterpret_cast<uint64_t*>(smem + (size_t)NST * Cfg::STAGE_BYTES + Cfg::RED_BYTES + 2 * Cfg::HALO_BYTES);
  const int tid = threadIdx.x;
  const int rl = 2 * (tid & 31);
  const int g = tid >> 5;
  const int dy0 = g * PER - P;
  const int tpr = wt_tiles_per_row(nx);
  const long long mine = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;  // tiles of this CTA
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) mbar_init(smem_addr(&bars[s]), 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0 && issue)
    for (int s = 0; s < NST && s < mine; ++s) {
      const long long t = blockIdx.x + (long long)s * gridDim.x;
      mbar_expect_tx(smem_addr(&bars[s]), Cfg::STAGE_BYTES);
      bulk_load(smem_addr(stages + (size_t)s * (Cfg::STAGE_BYTES / 4)), Wt + (size_t)t * (Cfg::STAGE_BYTES / 4),
                Cfg::STAGE_BYTES, smem_addr(&bars[s]));
    }
  if (mine > 0) load_halo<P, G>(halo, x, xb, yb, (int)(blockIdx.x / tpr), (int)(blockIdx.x % tpr), nx, ny);
  for (long long k = 0; k < mine; ++k) {
    const int s = (int)(k % NST);
    const bool ok = mbar_wait_bounded(smem_addr(&bars[s]), (uint32_t)((k / NST) & 1), wait_limit);
    cp_async_wait_all();  // this thread's halo copies of tile k
    if (__syncthreads_or(!ok)) {
      // give up: report, then let the copies still in flight land (bounded) before leaving
      if (tid == 0) {
        atomicExch(err, 1);
        for (long long j = k; j < mine && j < k + NST; ++j)
          mbar_wait_bounded(smem_addr(&bars[j % NST]), (uint32_t)((j / NST) & 1), wait_limit);
      }
      __syncthreads();
      return;
    }
    const long long tile = blockIdx.x + k * gridDim.x;
    const int iy = (int)(tile / tpr), bxi = (int)(tile % tpr);
    if (k + 1 < mine) {  // halo of the next tile into the other buffer (last read two tiles ago)
      const long long tn = tile + gridDim.x;
      load_halo<P, G>(halo + (size_t)((k + 1) & 1) * (Cfg::HALO_BYTES / 8), x, xb, yb, (int)(tn / tpr),
                      (int)(tn % tpr), nx, ny);
    }
    const int ix = bxi * R + rl;  // rows ix, ix + 1
    float2 aS[2] = {splat(0.f), splat(0.f)}, aT[2] = {splat(0.f), splat(0.f)};
    if (ix < nx) {
      const float2* hb = halo + (size_t)(k & 1) * (Cfg::HALO_BYTES / 8);
      const float4* cb = reinterpret_cast<const float4*>(hb + Cfg::XH);  // rows ix, ix + 1 (zero beyond nx)
      float2 b0[PW], b1[PW];
#pragma unroll
      for (int j = 0; j < PW / 2; ++j) {
        const float4 v0 = cb[(2 * j) * (R / 2) + (tid & 31)], v1 = cb[(2 * j + 1) * (R / 2) + (tid & 31)];
        b0[2 * j] = make_float2(v0.x, v0.y);
        b0[2 * j + 1] = make_float2(v0.z, v0.w);
        b1[2 * j] = make_float2(v1.x, v1.y);
        b1[2 * j + 1] = make_float2(v1.z, v1.w);
      }
      const float2* by = hb + Cfg::XH + Cfg::CB;
      float2 cyv[PER];
#pragma unroll
      for (int t = 0; t < PER; ++t) {  // {S_y, K_y}(iy, iy + dy): zero where iy + dy is outside the grid
        const int dy = dy0 + t;
        cyv[t] = dy <= P ? by[dy + P] : splat(0.f);
      }
      const float* w = stages + (size_t)s * (Cfg::STAGE_BYTES / 4) + rl;
      stencil_pair<P, G, PER>(hb + rl, w, cyv, b0, b1, dy0, aS, aT);
    }
    float4 part = make_float4(aS[0].x - tau * aT[0].y, aS[0].y + tau * aT[0].x, aS[1].x - tau * aT[1].y,
                              aS[1].y + tau * aT[1].x);
    float4* rb = reinterpret_cast<float4*>(red + (size_t)(k & 1) * (G - 1) * R);
    if (g > 0) rb[(g - 1) * (R / 2) + (tid & 31)] = part;
    __syncthreads();  // stage s and halo k consumed, partial sums visible
    if (tid == 0 && k + NST < mine) {
      const long long t = tile + (long long)NST * gridDim.x;
      mbar_expect_tx(smem_addr(&bars[s]), Cfg::STAGE_BYTES);
      bulk_load(smem_addr(stages + (size_t)s * (Cfg::STAGE_BYTES / 4)), Wt + (size_t)t * (Cfg::STAGE_BYTES / 4),
                Cfg::STAGE_BYTES, smem_addr(&bars[s]));
    }
    if (g == 0 && ix < nx) {
#pragma unroll
      for (int hh = 0; hh < G - 1; ++hh) {
        const float4 o = rb[hh * (R / 2) + (tid & 31)];
        part.x += o.x;
        part.y += o.y;
        part.z += o.z;
        part.w += o.w;
      }
      float2* yr = y + (long long)iy * nx + ix;
      yr[0] = make_float2(part.x, part.y);
      if (ix + 1 < nx) yr[1] = make_float2(part.z, part.w);
    }
  }
}

// ------------------------------------------------------------------------------- fast diagonalisation
// interleaved complex state (n0 x n1 x n2, x fastest) <-> two planar planes (re, then im) on the
// padded grid np0 x np1 x np2 (each axis rounded up to a multiple of 8 so that every GEMM leading
// dimension is 32-byte aligned); padding entries are zero
struct PadDims {
  int dim, n[3], np[3];
  long long Np;  // padded size of one plane (below 2^31: the index arithmetic below is 32-bit)
};
// padded plane index -> axis indices (j0 fastest)
__device__ __forceinline__ void pad_index(const PadDims& d, unsigned i, int& j0, int& j1, int& j2) {
  const unsigned n0 = (unsigned)d.np[0];
  const unsigned t = i / n0;
  j0 = (int)(i - t * n0);
  if (d.dim > 1) {
    const unsigned n1 = (unsigned)d.np[1];
    const unsigned u = t / n1;
    j1 = (int)(t - u * n1);
    j2 = (int)u;
  } else {
    j1 = 0;
    j2 = 0;
  }
}
// state index -> padded plane index
__device__ __forceinline__ unsigned pad_of_state(const PadDims& d, unsigned i) {
  const unsigned n0 = (unsigned)d.n[0];
  const unsigned t = i / n0;
  const unsigned j0 = i - t * n0;
  unsigned j1 = 0, j2 = 0;
  if (d.dim > 1) {
    const unsigned n1 = (unsigned)d.n[1];
    j2 = t / n1;
    j1 = t - j2 * n1;
  }
  return (j2 * (unsigned)d.np[1] + j1) * (unsigned)d.np[0] + j0;
}
template <class Tv, class Tp>
__global__ void k_split(const C<Tv>* __restrict__ v, Tp* __restrict__ w, PadDims d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d.Np; i += (long long)gridDim.x * blockDim.x) {
    int j0, j1, j2;
    pad_index(d, (unsigned)i, j0, j1, j2);
    const bool in = j0 < d.n[0] && (d.dim < 2 || j1 < d.n[1]) && (d.dim < 3 || j2 < d.n[2]);
    if (in) {
      const C<Tv> a = v[((long long)j2 * d.n[1] + j1) * d.n[0] + j0];
      w[i] = (Tp)a.r;
      w[d.Np + i] = (Tp)a.i;
    } else {
      w[i] = (Tp)0;
      w[d.Np + i] = (Tp)0;
    }
  }
}
template <class Tv, class Tp>
__global__ void k_merge(const Tp* __restrict__ w, C<Tv>* __restrict__ v, PadDims d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long k = pad_of_state(d, (unsigned)i);
    v[i] = C<Tv>{(Tv)w[k], (Tv)w[d.Np + k]};
  }
}
// k_merge that also accumulates the bilinear product res[0..1] += sum a_i v_i (binary64) of the merged
// vector with `a` (the preconditioned residual's rho = r^T z of COCG, without another pass)
template <class Tv, class Tp>
__global__ void k_merge_dot(const Tp* __restrict__ w, C<Tv>* __restrict__ v, PadDims d, long long n,
                            const C<Tv>* __restrict__ a, double* res, GridRed gr) {
  __shared__ double sh[32];
  double re = 0.0, im = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long k = pad_of_state(d, (unsigned)i);
    const C<Tv> z = C<Tv>{(Tv)w[k], (Tv)w[d.Np + k]};
    v[i] = z;
    const C<Tv> x = a[i];
    re += (double)x.r * (double)z.r - (double)x.i * (double)z.i;
    im += (double)x.r * (double)z.i + (double)x.i * (double)z.r;
  }
  re = block_sum(re, sh);
  im = block_sum(im, sh);
  const double sums[2] = {re, im};
  grid_reduce<2>(sums, res, gr, sh);
}

// k_split for the tensor-core transforms: each value as the TF32 pair (hi, lo), hi = the value rounded
// to TF32, lo = the FP32 remainder; planes of hi in whi, of lo in wlo
__global__ void k_split_tf32(const C<float>* __restrict__ v, float* __restrict__ whi, float* __restrict__ wlo,
                             PadDims d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d.Np; i += (long long)gridDim.x * blockDim.x) {
    int j0, j1, j2;
    pad_index(d, (unsigned)i, j0, j1, j2);
    const bool in = j0 < d.n[0] && (d.dim < 2 || j1 < d.n[1]) && (d.dim < 3 || j2 < d.n[2]);
    C<float> a{0.f, 0.f};
    if (in) a = v[((long long)j2 * d.n[1] + j1) * d.n[0] + j0];
    const float hr = tf32_hi(a.r), hi = tf32_hi(a.i);
    whi[i] = hr;
    whi[d.Np + i] = hi;
    wlo[i] = a.r - hr;
    wlo[d.Np + i] = a.i - hi;
  }
}

// in the eigenbasis (index j0 fastest): u /= 1 + i tm (lam0[j0] + lam1[j1] + lam2[j2]); binary64
template <class Tp>
// shifted = 1 (ground-state inverse iteration): 1 / (i (tm lam - ts)) instead, the inverse of the
// separable operator i tau (mbar K - sigma S) with ts = tau sigma
__global__ void k_fd_scale(Tp* __restrict__ w, long long n, int dim, int n0, int n1, const double* __restrict__ l0,
                           const double* __restrict__ l1, const double* __restrict__ l2, double tm, int shifted,
                           double ts) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int j0 = (int)(i % n0);
    const long long t = i / n0;
    double lam = l0[j0];
    if (dim > 1) lam += l1[(int)(t % n1)];
    if (dim > 2) lam += l2[(int)(t / n1)];
    const double th = tm * lam;
    const double a = (double)w[i], b = (double)w[n + i];
    if (shifted) {  // (a + i b) / (i d) = (b - i a) / d; a zero d (a padding entry at sigma = 0) gives 0
      const double d = th - ts, id = d != 0.0 ? 1.0 / d : 0.0;
      w[i] = (Tp)(b * id);
      w[n + i] = (Tp)(-a * id);
    } else {
      const double g = 1.0 / (1.0 + th * th);
      w[i] = (Tp)((a + th * b) * g);
      w[n + i] = (Tp)((b - th * a) * g);
    }
  }
}

// the same scaling in FP32 (eigenvalues in FP32), in place; the mixed preconditioner runs in FP32
// (shifted, ts: the ground-state scaling 1 / (i (tm lam - ts)), as in k_fd_scale)
__global__ void k_fd_scale32(float* __restrict__ w, PadDims d, const float* __restrict__ l0,
                             const float* __restrict__ l1, const float* __restrict__ l2, float tm, int shifted,
                             float ts) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d.Np; i += (long long)gridDim.x * blockDim.x) {
    int j0, j1, j2;
    pad_index(d, (unsigned)i, j0, j1, j2);
    float lam = l0[j0];
    if (d.dim > 1) lam += l1[j1];
    if (d.dim > 2) lam += l2[j2];
    const float th = tm * lam;
    const float a = w[i], b = w[d.Np + i];
    if (shifted) {
      const float dd = th - ts, id = dd != 0.0f ? 1.0f / dd : 0.0f;
      w[i] = b * id;
      w[d.Np + i] = -a * id;
    } else {
      const float g = 1.0f / fmaf(th, th, 1.0f);
      w[i] = fmaf(th, b, a) * g;
      w[d.Np + i] = fmaf(-th, a, b) * g;
    }
  }
}

// k_fd_scale32 for the tensor-core transforms: reads the FP32 planes w, writes the scaled values as
// TF32 pairs (planes of hi in whi, of lo in wlo)
__global__ void k_fd_scale_tf32(const float* __restrict__ w, float* __restrict__ whi, float* __restrict__ wlo,
                                PadDims d, const float* __restrict__ l0, const float* __restrict__ l1,
                                const float* __restrict__ l2, float tm, int shifted, float ts) {
  const long long n = d.Np;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int j0, j1, j2;
    pad_index(d, (unsigned)i, j0, j1, j2);
    float lam = l0[j0];
    if (d.dim > 1) lam += l1[j1];
    if (d.dim > 2) lam += l2[j2];
    const float th = tm * lam;
    const float a = w[i], b = w[n + i];
    float xr, xi;
    if (shifted) {
      const float dd = th - ts, id = dd != 0.0f ? 1.0f / dd : 0.0f;
      xr = b * id;
      xi = -a * id;
    } else {
      const float g = 1.0f / fmaf(th, th, 1.0f);
      xr = fmaf(th, b, a) * g;
      xi = fmaf(-th, a, b) * g;
    }
    const float hr = tf32_hi(xr), hi = tf32_hi(xi);
    whi[i] = hr;
    whi[n + i] = hi;
    wlo[i] = xr - hr;
    wlo[n + i] = xi - hi;
  }
}

}  // namespace nd
}  // namespace tdz

// ================================================================================= host driver
using namespace tdz;
using namespace tdz::nd;

namespace {

int nd_cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return TDZ_ECUDA;
}

// grid of the row kernels: x over a row's `width` outputs, y over rows (grid-stride), about 16 blocks per SM
inline dim3 row_grid(int width, long long rows) {
  const int gx = (width + TPB - 1) / TPB;
  const long long gy = std::max<long long>(1, std::min<long long>({rows, 65535LL, (148LL * 16 + gx - 1) / gx}));
  return dim3((unsigned)gx, (unsigned)gy);
}

constexpr size_t kFusedStageMax = 72 * 1024;  // shared-memory tables of k_fused_last: three blocks per SM

inline int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + TPB - 1) / TPB, 148 * 16)); }

// element chunks of the fused last-axis passes: enough threads (about 150k) over the pencils, each
// chunk at least 2P+2 elements long
inline long long fused_nchunks(int E, long long inner, int P, int* echunk) {
  long long nch = std::max<long long>(1, std::min<long long>(E / (2 * P + 2), (150000 + inner - 1) / inner));
  const int ec = (int)((E + nch - 1) / nch);
  *echunk = ec;
  return (E + ec - 1) / ec;
}

// element chunks of the observables pass: as many blocks of 256 as fill one to three whole waves of
// its three resident blocks per SM (the fewest idle slots in the last wave), each chunk at least 2P+2
// elements long
inline long long reduce_nchunks(int E, long long inner, int P, int* echunk) {
  const long long wave = 148LL * 3 * 256, nmax = std::max(1, E / (2 * P + 2));
  long long best = 1;
  double best_fill = -1.0;
  for (int m = 1; m <= 3; ++m) {
    const long long nch = std::max<long long>(1, std::min<long long>(nmax, m * wave / inner));
    const int ec = (int)((E + nch - 1) / nch);
    const long long n = (E + ec - 1) / ec;
    const long long thr = ((inner * n + 255) / 256) * 256;
    const double fill = (double)thr / (double)(((thr + wave - 1) / wave) * wave);
    if (fill >= best_fill) {
      best_fill = fill;
      best = n;
    }
  }
  *echunk = (int)((E + best - 1) / best);
  return (E + *echunk - 1) / *echunk;
}

struct NdRun {
  int ops = 0;
  int dim = 0, P = 0;
  long long N = 0;
  int n[3] = {0, 0, 0}, E[3] = {0, 0, 0}, nq[3] = {0, 0, 0}, Q[3] = {0, 0, 0};
  AxisDev ax[3];
  MediumDev med;
  int geo = 0;          // index of the geometry tables (fast diagonalisation, stencil)
  bool const_mass = true;
  bool cap = false;     // the geometry has an absorbing layer (tau W_a terms in the Kronecker pass)
  double cm = 1.0;      // m^-1 for constant mass
  double mbar = 1.0;    // mean m^-1 for the preconditioner
  double2* c = nullptr;  // state, binary64
  int status = TDZ_OK;
  double max_rel = 0.0;
  long long nsolve = 0;
  long long iters = 0;
};

}  // namespace

namespace tdz {

// per geometry: fast-diagonalisation factors (S-orthonormal eigenvectors, column j = vector j, and
// eigenvalues) and the assembled 2-D stencil
struct NdGeo {
  bool fd = false;
  int n[3] = {0, 0, 0};
  int np[3] = {1, 1, 1};  // n rounded up to a multiple of 8 (fast-diagonalisation work layout)
  double* V64[3] = {nullptr, nullptr, nullptr};
  // mixed batches: V rounded to TF32 once, as the tensor-core transforms read it: Vt row j = eigenvector
  // j (the forward transform V^T), VtT = its transpose (the inverse transform V)
  float* Vt[3] = {nullptr, nullptr, nullptr};
  float* VtT[3] = {nullptr, nullptr, nullptr};
  float* lam32[3] = {nullptr, nullptr, nullptr};  // the eigenvalues in FP32 (mixed batches)
  // transform variant chosen by the autotuner: bit 0 = 256-column tiles (else 128), bit 1 = the data
  // split into TF32 pairs in shared memory by the transform (else by the producing kernels, as pairs
  // in memory); -1 = not tuned
  int tc_variant = -1;
  float tc_ms[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // the autotuner's ms per preconditioner apply of variants 0..5
  double* lam[3] = {nullptr, nullptr, nullptr};
  double* W64 = nullptr;  // binary64 batches
  float* W32 = nullptr;   // mixed: inner FP32 solve
  fx* Wx = nullptr;       // mixed: double-float residual
  bool has_stencil() const { return W64 || W32; }
  int apply_groups = 8;  // variant of the fused FP32 2-D apply (groups of offsets dy per row)
  float tune_ms[2] = {0.f, 0.f};  // autotuner timings of the variants G = 8, 16 (ms per apply)
  // 3-D mixed: w V at the Gauss points ([q_z][q_y][q_x]) for the FP32 and double-float passes
  fx* Vqx = nullptr;
  fx* Gq = nullptr;  // soft-core observables' point factor (double-float), or null (evaluated per point)
};

struct NdBatch {
  int prec = TDZ_FP64;
  int dim = 0;
  int P = 0;
  int nruns = 0;
  cudaStream_t st = nullptr;
  std::vector<NdRun> runs;
  std::vector<Ops> ops;  // copies of the operators (per-axis factors for the preconditioner)
  std::vector<NdGeo> geo;
  cublasHandle_t blas = nullptr;
  int opt_precond = TDZ_PRECOND_AUTO;
  int opt_operator = TDZ_OPERATOR_AUTO;
  int opt_groups = 0;  // fused 2-D apply variant: 0 = the autotuned one, else 8 or 16 groups
  int opt_wait_test = 0;  // test aid: the fused 2-D apply issues no copies and its waits run out
  std::vector<void*> bufs;
  // work vectors sized for the largest run: binary64 and solve precision
  size_t maxN = 0, maxQ = 0;
  double2 *d_r0 = nullptr, *d_y = nullptr, *d_t1 = nullptr, *d_t2 = nullptr, *d_t3 = nullptr, *d_t4 = nullptr;
  double2 *d_qa = nullptr, *d_qb = nullptr;
  double2 *d_z = nullptr, *d_p = nullptr, *d_q = nullptr, *d_rc = nullptr;  // COCG / residual vectors
  void *w_x = nullptr, *w_r = nullptr, *w_z = nullptr, *w_p = nullptr, *w_q = nullptr, *w_t1 = nullptr, *w_t2 = nullptr,
       *w_t3 = nullptr, *w_t4 = nullptr, *w_qa = nullptr, *w_qb = nullptr;
  void *w_qc = nullptr, *w_qd = nullptr;  // mixed: second TF32 pair of the fast-diagonalisation transforms
  size_t maxPad = 0;                      // largest padded plane of a run (fast diagonalisation)
  void* pre_L[3] = {nullptr, nullptr, nullptr};  // per run would be needed for different sizes; refreshed per run
  void* pre_D[3] = {nullptr, nullptr, nullptr};
  double* d_red = nullptr;  // reduction scratch (16 doubles)
  GridRed gr{};             // per-block partial sums of the fixed-order reductions
  int* d_err = nullptr;     // set to nonzero by a kernel whose bounded wait ran out (in d_red's last slot)
  bool wait_failed = false;  // host copy of *d_err as of the last reduction read
  // coefficient rows {S, K} of the separable part for the fused FP32 2-D apply (x and y axes), and
  // what they were computed for: geometry, Ebar_x, Ebar_y, constant-mass m^-1
  float2* rb32[2] = {nullptr, nullptr};
  int rb_geo = -1;
  double rb_key[3] = {0, 0, 0};
  int nsm = 148;  // SM count of the device (persistent grids)
  std::string dev_name;  // the device's name (autotuner cache keys)
  void* d_side = nullptr;   // chunk-boundary partial sums of the fused last-axis pass
  size_t maxSide = 0;
  int maxn = 0;
  size_t work_bytes = 0;  // device bytes of one worker's work buffers
  // batches of several runs: extra workers (own stream, cuBLAS handle and work buffers; geometry
  // tables and run states shared with this batch) that propagate runs concurrently
  std::vector<NdBatch*> workers;
  bool own_stream = false;
  std::vector<double> obs;  // host copy [run][nsteps][2+3dim]
  long long last_nsteps = 0;
  double tol = 1e-12;
  int max_it = 400;
  double inner_tol = 1e-6;
  // ground-state inverse iteration (binary64 batches): the operator and the preconditioner of the
  // worker's Krylov solves become those of A - (1 + i tau sigma) S = i tau (H0 - sigma S)
  bool eig = false;
  double eig_sigma = 0.0;
  size_t dev_bytes = 0;

  void* alloc(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    cudaMemsetAsync(p, 0, bytes, st);
    bufs.push_back(p);
    dev_bytes += bytes;
    return p;
  }
  ~NdBatch() {
    for (NdBatch* w : workers) delete w;
    if (blas) cublasDestroy(blas);
    for (void* p : bufs) cudaFree(p);
    if (own_stream && st) cudaStreamDestroy(st);
  }
};

}  // namespace tdz

namespace {

// ---------------------------------------------------------------- operator application (templated)
// y = A_n x through the fused TMA-fed 2-D kernel (FP32) with G groups of offsets dy per row
template <int P, int G>
void launch_apply2d(NdBatch* b, const NdRun* r, const float* Wt, const float2* x, float2* y, double tau) {
  using Cfg = Apply2dCfg<P, G>;
  cudaFuncSetAttribute(k_apply2d_tma<P, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
  const long long ntiles = (long long)r->n[1] * wt_tiles_per_row(r->n[0]);
  const int grid = (int)std::min<long long>(ntiles, b->nsm);
  const long long limit = b->opt_wait_test ? kWaitLimitTest : kWaitLimit;
  k_apply2d_tma<P, G><<<grid, Cfg::THREADS, Cfg::SMEM, b->st>>>(Wt, ntiles, x, y, b->rb32[0], b->rb32[1], r->n[0],
                                                                r->n[1], (float)tau, b->d_err, limit,
                                                                b->opt_wait_test ? 0 : 1);
}

// refresh the per-axis coefficient rows when the geometry or the field changed, then one
// persistent launch over the stencil tiles in the variant chosen for this geometry
template <int P>
void apply2d_fused(NdBatch* b, NdRun* r, const float* Wt, const C<float>* x, C<float>* y, double tau,
                   const double* ebar) {
  constexpr int PW = 2 * P + 2;
  const double cm = r->const_mass ? r->cm : 0.0;
  if (b->rb_geo != r->geo || b->rb_key[0] != ebar[0] || b->rb_key[1] != ebar[1] || b->rb_key[2] != cm) {
    for (int a = 0; a < 2; ++a) {
      const AxisDev& A = r->ax[a];
      k_rowband<P><<<grid_for((long long)A.n * PW), TPB, 0, b->st>>>(A.fS, A.fT1, A.fD, A.n, (float)cm,
                                                                    (float)ebar[a], b->rb32[a]);
    }
    b->rb_geo = r->geo;
    b->rb_key[0] = ebar[0];
    b->rb_key[1] = ebar[1];
    b->rb_key[2] = cm;
  }
  const float2* xv = reinterpret_cast<const float2*>(x);
  float2* yv = reinterpret_cast<float2*>(y);
  const int groups = b->opt_groups ? b->opt_groups : b->geo[r->geo].apply_groups;
  if (groups == 16) launch_apply2d<P, 16>(b, r, Wt, xv, yv, tau);
  else launch_apply2d<P, 8>(b, r, Wt, xv, yv, tau);
}

// Autotuner of the fused FP32 2-D apply: every variant is timed on this batch's own work buffers
// (CUDA events on the batch stream, one warm-up launch, then the best of three) for the first run
// of each geometry with a stencil, and the fastest is kept for that geometry.
template <int P>
int autotune_apply2d(NdBatch* b) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return TDZ_ECUDA;
  }
  const int cand[2] = {8, 16};
  const double zero[3] = {0.0, 0.0, 0.0};
  const double tau = 0.025;
  int rc = TDZ_OK;
  for (size_t g = 0; g < b->geo.size() && rc == TDZ_OK; ++g) {
    NdGeo& G = b->geo[g];
    NdRun* r = nullptr;
    for (auto& run : b->runs)
      if (run.geo == (int)g) {
        r = &run;
        break;
      }
    if (!G.W32 || !r || r->cap) continue;  // an absorbing layer takes the unfused apply
    const std::string key = "apply2d p=" + std::to_string(P) + " n=" + std::to_string(r->n[0]) + "," +
                            std::to_string(r->n[1]) + " mixed dev=" + b->dev_name;
    std::vector<double> hit;
    if (tune_cache_get(key, hit) && hit.size() == 3 && (hit[0] == 8 || hit[0] == 16)) {
      G.apply_groups = (int)hit[0];
      G.tune_ms[0] = (float)hit[1];
      G.tune_ms[1] = (float)hit[2];
      continue;
    }
    const C<float>* x = static_cast<const C<float>*>(b->w_p);
    C<float>* y = static_cast<C<float>*>(b->w_q);
    for (int c = 0; c < 2; ++c) {
      G.apply_groups = cand[c];
      apply2d_fused<P>(b, r, G.W32, x, y, tau, zero);
      float tmin = 0.f;
      for (int k = 0; k < 3; ++k) {
        cudaEventRecord(e0, b->st);
        apply2d_fused<P>(b, r, G.W32, x, y, tau, zero);
        cudaEventRecord(e1, b->st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          rc = TDZ_ECUDA;
          break;
        }
        tmin = k == 0 ? ms : std::min(tmin, ms);
      }
      G.tune_ms[c] = tmin;
    }
    G.apply_groups = G.tune_ms[1] < G.tune_ms[0] ? 16 : 8;
    if (rc == TDZ_OK) tune_cache_put(key, {(double)G.apply_groups, (double)G.tune_ms[0], (double)G.tune_ms[1]});
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->rb_geo = -1;
  int werr = 0;  // a wait that ran out while timing
  if (rc == TDZ_OK && (cudaMemcpy(&werr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || werr != 0))
    rc = TDZ_ECUDA;
  return rc;
}

int autotune(NdBatch* b) {
  switch (b->P) {
    case 1: return autotune_apply2d<1>(b);
    case 2: return autotune_apply2d<2>(b);
    case 3: return autotune_apply2d<3>(b);
    case 4: return autotune_apply2d<4>(b);
    case 5: return autotune_apply2d<5>(b);
    case 6: return autotune_apply2d<6>(b);
    case 7: return autotune_apply2d<7>(b);
    default: return autotune_apply2d<8>(b);
  }
}

template <class T, int P>
struct Apply {
  NdBatch* b;
  NdRun* r;
  C<T>* t1;
  C<T>* t2;
  C<T>* t3;
  C<T>* t4;
  C<T>* qa;
  C<T>* qb;
  const T* Wm = nullptr;  // assembled 2-D stencil of the non-separable terms, or null (quadrature)
  const T* Vtab = nullptr;  // w V at the Gauss points (3-D), or null (evaluated per point)
  // double-float only: when set, the next potential-term pass also reduces c^H G_a c of its input into
  // obs_res[0..3) (k_fused_last_fx<P, true>; obs_gtab = the soft-core point factor); cleared by that pass
  const fx* obs_gtab = nullptr;
  double* obs_res = nullptr;

  // shape helpers: lengths of axes with the first `k` axes already in quadrature space
  void shape(int axis, const int* len, long long& outer, long long& inner) const {
    inner = 1;
    outer = 1;
    for (int a = 0; a < axis; ++a) inner *= len[a];
    for (int a = axis + 1; a < r->dim; ++a) outer *= len[a];
  }

  // out = sum over Kronecker terms: factors per axis f[a] applied to input; generic two-stream scheme
  // out = [S_z] [S_y] (S_x + i tau K_x) x + i tau [S_z] K_y S_x x + i tau K_z S_y S_x x   (3-D)
  // with K_a = cm T1_a + Ebar_a D_a - i W_a (the absorbing layer's axis factor W_a, when present, enters
  // as the real term tau W_a). Mode "S only": out = (x)S x. Mode "D_a": D_a on axis a, S elsewhere.
  void kron(const C<T>* x, C<T>* out, int mode, double tau, const double* ebar, int daxis = 0) {
    const int D = r->dim;
    int len[3] = {r->n[0], r->n[1], r->n[2]};
    // streams: a = S-product so far, bsum = accumulated operator
    const C<T>* a_in = x;
    const C<T>* b_in = x;
    C<T>* bufs[4] = {t1, t2, t3, t4};
    int nb = 0;
    for (int ax = 0; ax < D; ++ax) {
      long long outer, inner;
      shape(ax, len, outer, inner);
      const AxisDev& A = r->ax[ax];
      const bool last = ax == D - 1;
      C<T>* a_out = last ? nullptr : bufs[nb++ % 4];
      C<T>* b_out = last ? out : bufs[nb++ % 4];
      BandTerms<T> ta{}, tb{};
      if (mode == 0) {  // A_sep
        // a stream: S_ax a
        ta.nt = 1;
        ta.R[0] = tab<T>(A, TS);
        ta.cr[0] = 1;
        ta.ci[0] = 0;
        ta.sel[0] = 0;
        // b stream: S_ax b + i tau K_ax a  (for the first axis a == b == x)
        tb.nt = 3;
        tb.R[0] = tab<T>(A, TS);
        tb.cr[0] = 1;
        tb.ci[0] = 0;
        tb.sel[0] = 1;
        tb.R[1] = tab<T>(A, TT1);
        tb.cr[1] = 0;
        tb.ci[1] = tau * (r->const_mass ? r->cm : 0.0);
        tb.sel[1] = 0;
        tb.R[2] = tab<T>(A, TD);
        tb.cr[2] = 0;
        tb.ci[2] = tau * ebar[ax];
        tb.sel[2] = 0;
        if (r->cap) {
          tb.nt = 4;
          tb.R[3] = tab<T>(A, TCAP);
          tb.cr[3] = tau;
          tb.ci[3] = 0;
          tb.sel[3] = 0;
        }
      } else if (mode == 1) {  // S only
        ta.nt = 1;
        ta.R[0] = tab<T>(A, TS);
        ta.cr[0] = 1;
        ta.sel[0] = 0;
        tb = ta;
      } else {  // D on daxis, S elsewhere
        ta.nt = 1;
        ta.R[0] = ax == daxis ? tab<T>(A, TD) : tab<T>(A, TS);
        ta.cr[0] = 1;
        ta.sel[0] = 0;
        tb = ta;
      }
      const long long tot = outer * len[ax] * inner;
      if (!last && mode == 0)
        launch_axis_band<T, P>(b->st, grid_for(tot), ta, a_in, b_in, a_out, outer, len[ax], inner);
      if (mode == 0) {
        launch_axis_band<T, P>(b->st, grid_for(tot), tb, a_in, b_in, b_out, outer, len[ax], inner);
      } else {
        launch_axis_band<T, P>(b->st, grid_for(tot), tb, b_in, b_in, b_out, outer, len[ax], inner);
      }
      if (!last && mode == 0) a_in = a_out;
      b_in = b_out;
    }
  }

  QGrid<T> grid() const {
    QGrid<T> g{};
    g.dim = r->dim;
    for (int a = 0; a < r->dim; ++a) {
      g.Q[a] = r->Q[a];
      g.x[a] = tab<T>(r->ax[a], TX);
      g.w[a] = tab<T>(r->ax[a], TW);
    }
    return g;
  }

  // interpolate x along the faster axes 0..dim-2 (derivative on axis dax if dax < dim - 1); returns the
  // result (shape [n_last][Q_0..Q_{dim-2}]) in qa or qb
  // one interpolation / projection pass along an axis: the sliding-window kernels where the inner
  // extent is contiguous enough to coalesce, else one thread per output
  void interp(const T* B, const AxisDev& A, const C<T>* in, C<T>* out, long long outer, long long inner) {
    if (inner >= 32)
      k_interp_win<T, P><<<grid_for(outer * inner), TPB, 0, b->st>>>(B, A.nq, A.n, A.E, in, out, outer, inner);
    else if (inner == 1)
      k_interp_row<T, P><<<row_grid(A.Q, outer), TPB, 0, b->st>>>(B, A.nq, A.n, A.Q, in, out, outer);
    else
      k_interp<T, P><<<grid_for(outer * A.Q * inner), TPB, 0, b->st>>>(B, A.nq, A.n, A.Q, in, out, outer, inner);
  }
  void project(const T* B, const AxisDev& A, const C<T>* in, C<T>* out, long long outer, long long inner, int acc) {
    if (inner >= 32)
      k_project_win<T, P><<<grid_for(outer * inner), TPB, 0, b->st>>>(B, A.nq, A.n, A.E, in, out, outer, inner, acc);
    else if (inner == 1)
      k_project_row<T, P><<<row_grid(A.n, outer), TPB, 0, b->st>>>(B, A.nq, A.n, A.E, in, out, outer, acc);
    else
      k_project<T, P><<<grid_for(outer * A.n * inner), TPB, 0, b->st>>>(B, A.nq, A.n, A.E, in, out, outer, inner, acc);
  }

  const C<T>* to_pencils(const C<T>* x, int dax) {
    const int D = r->dim, L = D - 1;
    int len[3] = {r->n[0], r->n[1], r->n[2]};
    const C<T>* in = x;
    for (int ax = 0; ax < L; ++ax) {
      long long outer, inner;
      shape(ax, len, outer, inner);
      const AxisDev& A = r->ax[ax];
      C<T>* X = (ax % 2 == 0) ? qa : qb;
      interp(tab<T>(A, ax == dax ? TDB : TB), A, in, X, outer, inner);
      len[ax] = A.Q;
      in = X;
    }
    return in;
  }

  // y += coef * (Gauss-point operator of kind `kind`) x, derivative on axis dax (or none if dax < 0):
  // interpolate along the faster axes, fused interpolate/multiply/project along the last axis,
  // project back along the faster axes.
  void quad(const C<T>* x, C<T>* y, int dax, int kind, int faxis, double cr, double ci) {
    const int D = r->dim, L = D - 1;
    int len[3] = {r->n[0], r->n[1], r->n[2]};
    const C<T>* in = x;
    C<T>* X = nullptr;
    for (int ax = 0; ax < L; ++ax) {
      long long outer, inner;
      shape(ax, len, outer, inner);
      const AxisDev& A = r->ax[ax];
      X = (ax % 2 == 0) ? qa : qb;
      interp(tab<T>(A, ax == dax ? TDB : TB), A, in, X, outer, inner);
      len[ax] = A.Q;
      in = X;
    }
    C<T>* U = (X == qa) ? qb : qa;
    long long inner = 1;
    for (int a = 0; a < L; ++a) inner *= len[a];
    const AxisDev& AL = r->ax[L];
    int echunk = 1;
    const long long nch = fused_nchunks(AL.E, inner, P, &echunk);
    C<T>* side = static_cast<C<T>*>(b->d_side);
    const T* ftab = (kind == 0 && dax < 0 && D == 3) ? Vtab : nullptr;
    // stage the last axis' tables in shared memory when they fit three blocks per SM
    const size_t QL = (size_t)AL.E * AL.nq;
    const size_t tab_bytes = sizeof(T) * QL * (P + 1 + (ftab ? 0 : 2));
    const bool stage = tab_bytes <= kFusedStageMax;
    // raised once per instantiation (thread-safe static initialisation: the batch's workers share it)
    static const cudaError_t attr_set =
        cudaFuncSetAttribute(k_fused_last<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedStageMax);
    (void)attr_set;
    if constexpr (std::is_same<T, fx>::value) {
      const bool obs = obs_res && kind == 0 && dax < 0;
      if (obs)
        k_fused_last_fx<P, true><<<grid_for(inner * nch), TPB, 0, b->st>>>(
            in, U, side, tab<T>(AL, TB), AL.nq, AL.n, AL.E, inner, echunk, grid(), medium_t<T>(r->med), kind, faxis,
            cr, ci, ftab, obs_gtab, obs_res, b->gr);
      else
        k_fused_last_fx<P, false><<<grid_for(inner * nch), TPB, 0, b->st>>>(
            in, U, side, tab<T>(AL, L == dax ? TDB : TB), AL.nq, AL.n, AL.E, inner, echunk, grid(),
            medium_t<T>(r->med), kind, faxis, cr, ci, ftab, nullptr, nullptr, b->gr);
      if (obs) obs_res = nullptr, obs_gtab = nullptr;
    } else
      k_fused_last<T, P><<<grid_for(inner * nch), TPB, stage ? tab_bytes : 0, b->st>>>(
          in, U, side, tab<T>(AL, L == dax ? TDB : TB), AL.nq, AL.n, AL.E, inner, echunk, grid(),
          medium_t<T>(r->med), kind, faxis, cr, ci, ftab, stage ? 1 : 0);
    if (nch > 1)
      k_fused_fixup<T, P><<<grid_for((nch - 1) * P * inner), TPB, 0, b->st>>>(U, side, AL.n, inner, echunk, (int)nch);
    len[L] = AL.n;
    C<T>* cur = U;
    for (int ax = L - 1; ax >= 0; --ax) {
      long long outer2, inner2;
      shape(ax, len, outer2, inner2);
      const AxisDev& A = r->ax[ax];
      const bool last = ax == 0;
      C<T>* out = last ? y : ((cur == qa) ? qb : qa);
      project(tab<T>(A, ax == dax ? TDB : TB), A, cur, out, outer2, inner2, last ? 1 : 0);
      len[ax] = A.n;
      cur = out;
    }
  }

  // y = A_n x, or in a ground-state solve (binary64) y = A x - (1 + i tau sigma) S x = i tau (H0 - sigma S) x
  void apply(const C<T>* x, C<T>* y, double tau, const double* ebar) {
    apply_a(x, y, tau, ebar);
    if constexpr (!std::is_same<T, fx>::value) {
      if (b->eig) {  // (binary64 batch, or the FP32 solve of a mixed batch)
        double zero3[3] = {0, 0, 0};
        C<T>* s = reinterpret_cast<C<T>*>(b->d_rc);
        kron(x, s, 1, 0.0, zero3);
        k_caxpby<T><<<grid_for(r->N), TPB, 0, b->st>>>(s, y, r->N, -1.0, -tau * b->eig_sigma, 1.0, 0.0);
      }
    }
  }
  void apply_a(const C<T>* x, C<T>* y, double tau, const double* ebar) {
    if constexpr (std::is_same<T, float>::value) {
      if (Wm && r->dim == 2 && !r->cap) {  // FP32 2-D with the stencil: one fused pass (Kronecker terms + W)
        apply2d_fused<P>(b, r, Wm, x, y, tau, ebar);
        return;
      }
    }
    kron(x, y, 0, tau, ebar);
    if (Wm) {  // i tau (V + variable-mass kinetic) through the assembled stencil (half storage)
      k_wapply<T, P><<<grid_for(r->N), TPB, 0, b->st>>>(Wm, x, y, r->n[0], r->n[1], (T)tau);
      return;
    }
    if (r->med.pot_kind != TDZ_POT_ZERO) quad(x, y, -1, 0, 0, 0.0, tau);  // i tau V
    if (!r->const_mass)
      for (int a = 0; a < r->dim; ++a) quad(x, y, a, 1, a, 0.0, tau);     // i tau 1/2 <d_a| m^-1 |d_a>
  }
};

template <class T, int P>
void line_precond(NdBatch* b, NdRun* r, C<T>* v) {
  int len[3] = {r->n[0], r->n[1], r->n[2]};
  for (int ax = 0; ax < r->dim; ++ax) {
    long long inner = 1, outer = 1;
    for (int a = 0; a < ax; ++a) inner *= len[a];
    for (int a = ax + 1; a < r->dim; ++a) outer *= len[a];
    k_line_solve<T, P><<<grid_for(outer * inner), 128, 0, b->st>>>(v, static_cast<const C<T>*>(b->pre_L[ax]),
                                                                    static_cast<const C<T>*>(b->pre_D[ax]), outer,
                                                                    len[ax], inner);
  }
}

// ---------------------------------------------------------------- fast diagonalisation
inline PadDims pad_dims(const NdGeo& G, const NdRun* r) {
  PadDims d{};
  d.dim = r->dim;
  d.Np = 1;
  for (int a = 0; a < 3; ++a) {
    d.n[a] = a < r->dim ? r->n[a] : 1;
    d.np[a] = a < r->dim ? G.np[a] : 1;
    d.Np *= d.np[a];
  }
  return d;
}

// v <- M^-1 v, M = S(x)S + i tau mbar sum_a (T1_a on axis a, S elsewhere):
//   M^-1 = ((x)V_a) diag(1 / (1 + i tau mbar sum_a lam_a)) ((x)V_a)^T   since V_a^T S_a V_a = I,
//   V_a^T T1_a V_a = diag(lam_a). Both planes (re, im) are transformed together; sizes are padded to
//   multiples of 8 (zero entries), so every row is 32-byte aligned.
//
// Binary64 batches: one cuBLAS DGEMM per axis contracts the slowest axis of the current layout (length
// ns, R = N / ns values per index) with V^T (forward) or V (inverse) and writes the new index fastest:
//   out(j, r) = sum_k M(k, j) in(r, k), both planes as a batch of two.
inline cublasStatus_t gemm_rot(cublasHandle_t h, bool inv, int ns, int R, const double* V, const double* in,
                               double* out, long long stride) {
  const double one = 1.0, zero = 0.0;
  return cublasGemmStridedBatchedEx(h, inv ? CUBLAS_OP_N : CUBLAS_OP_T, CUBLAS_OP_T, ns, R, ns, &one, V, CUDA_R_64F, ns, 0,
                                    in, CUDA_R_64F, R, stride, &zero, out, CUDA_R_64F, ns, stride, 2, CUBLAS_COMPUTE_64F,
                                    CUBLAS_GEMM_DEFAULT);
}

// dst = M^-1 src (src == dst allowed); with dot, also dot[0..1] += src^T dst (src != dst).
// w0, w1: planar scratch of 2 Np values each.
void fd_apply64(NdBatch* b, const NdRun* r, const C<double>* src, C<double>* dst, double* w0, double* w1, double tau,
                double* dot) {
  const NdGeo& G = b->geo[r->geo];
  const PadDims d = pad_dims(G, r);
  k_split<double, double><<<grid_for(d.Np), TPB, 0, b->st>>>(src, w0, d);
  double* cur = w0;
  double* nxt = w1;
  for (int pass = 0; pass < 2; ++pass) {
    for (int a = r->dim - 1; a >= 0; --a) {
      const int ns = d.np[a];
      gemm_rot(b->blas, pass == 1, ns, (int)(d.Np / ns), G.V64[a], cur, nxt, d.Np);
      std::swap(cur, nxt);
    }
    if (pass == 0)
      k_fd_scale<double><<<grid_for(d.Np), TPB, 0, b->st>>>(cur, d.Np, r->dim, d.np[0], d.np[1], G.lam[0], G.lam[1],
                                                            G.lam[2], tau * r->mbar, b->eig ? 1 : 0,
                                                            tau * b->eig_sigma);
  }
  if (dot)
    k_merge_dot<double, double><<<grid_for(r->N), TPB, 0, b->st>>>(cur, dst, d, r->N, src, dot, b->gr);
  else
    k_merge<double, double><<<grid_for(r->N), TPB, 0, b->st>>>(cur, dst, d, r->N);
}

// Mixed batches: the transforms run on the tensor cores (tc_axis_transform). Each contracts the
// FASTEST axis of the current layout with the TF32-rounded factor (Vt forward, VtT inverse) and
// writes the new index slowest, so after one transform per axis the original order is back. The data
// enter every transform as a TF32 pair (hi, lo), either split by the transform itself in shared
// memory (FP32 planes in memory) or written as pairs by the split kernel, the eigenvalue scaling and
// every transform but the last of a pass (variant bit 1 clear). Rounding V once keeps
// M^-1 = Vt Lambda Vt^T complex symmetric, as COCG requires; it is the preconditioner of V rounded to
// 11 significant bits. w0..w3: planar scratch of 2 Np FP32 values each (w2, w3 only for pairs in
// memory). Returns TDZ_OK or the transform's error.
int fd_apply32(NdBatch* b, const NdRun* r, const C<float>* src, C<float>* dst, float* w0, float* w1, float* w2,
               float* w3, double tau, double* dot) {
  const NdGeo& G = b->geo[r->geo];
  const PadDims d = pad_dims(G, r);
  const int v = G.tc_variant < 0 ? 0 : G.tc_variant;
  const int tile = v >= 4 ? 64 : (v & 1) ? 256 : 128;  // variants 4, 5: 64-column tiles
  const bool smem_split = v >= 4 ? v == 5 : (v & 2) != 0;
  float* out = nullptr;  // the FP32 result of the last transform
  if (smem_split) {
    k_split<float, float><<<grid_for(d.Np), TPB, 0, b->st>>>(src, w0, d);
    float *cur = w0, *nxt = w1;
    for (int pass = 0; pass < 2; ++pass) {
      for (int a = 0; a < r->dim; ++a) {
        const int ns = d.np[a];
        const long long R = d.Np / ns;
        const int rc = tc_axis_transform(cur, nullptr, 2 * R, ns, pass == 0 ? G.Vt[a] : G.VtT[a], nullptr, ns, R, d.Np,
                                         nxt, nullptr, b->d_err, tile, b->st);
        if (rc != TDZ_OK) return rc;
        std::swap(cur, nxt);
      }
      if (pass == 0)
        k_fd_scale32<<<grid_for(d.Np), TPB, 0, b->st>>>(cur, d, G.lam32[0], G.lam32[1], G.lam32[2],
                                                        (float)(tau * r->mbar), b->eig ? 1 : 0,
                                                        (float)(tau * b->eig_sigma));
    }
    out = cur;
  } else {
    k_split_tf32<<<grid_for(d.Np), TPB, 0, b->st>>>(src, w0, w1, d);
    float *hi = w0, *lo = w1, *ohi = w2, *olo = w3;
    for (int pass = 0; pass < 2; ++pass) {
      for (int a = 0; a < r->dim; ++a) {
        const int ns = d.np[a];
        const long long R = d.Np / ns;
        const bool last = a == r->dim - 1;
        const int rc = tc_axis_transform(hi, lo, 2 * R, ns, pass == 0 ? G.Vt[a] : G.VtT[a], nullptr, ns, R, d.Np, ohi,
                                         last ? nullptr : olo, b->d_err, tile, b->st);
        if (rc != TDZ_OK) return rc;
        std::swap(hi, ohi);
        std::swap(lo, olo);
      }
      // hi holds the FP32 result of the pass
      if (pass == 0) {
        k_fd_scale_tf32<<<grid_for(d.Np), TPB, 0, b->st>>>(hi, ohi, olo, d, G.lam32[0], G.lam32[1], G.lam32[2],
                                                           (float)(tau * r->mbar), b->eig ? 1 : 0,
                                                           (float)(tau * b->eig_sigma));
        std::swap(hi, ohi);
        std::swap(lo, olo);
      }
    }
    out = hi;
  }
  if (dot)
    k_merge_dot<float, float><<<grid_for(r->N), TPB, 0, b->st>>>(out, dst, d, r->N, src, dot, b->gr);
  else
    k_merge<float, float><<<grid_for(r->N), TPB, 0, b->st>>>(out, dst, d, r->N);
  return TDZ_OK;
}

bool use_fd(const NdBatch* b, const NdRun* r) {
  return b->opt_precond != TDZ_PRECOND_LINES && b->geo[r->geo].fd;
}

// Autotuner of the mixed fast-diagonalisation preconditioner: one whole apply (split, 2 dim tensor-core
// transforms, scaling, merge) is timed in each of the four transform variants (128- or 256-column
// tiles; data split into TF32 pairs in shared memory or by the producing kernels) on the batch's own
// buffers (CUDA events, best of three after one warm-up) and the fastest is kept per geometry.
int autotune_fd(NdBatch* b) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return TDZ_ECUDA;
  }
  int rc = TDZ_OK;
  for (size_t g = 0; g < b->geo.size() && rc == TDZ_OK; ++g) {
    NdGeo& G = b->geo[g];
    NdRun* r = nullptr;
    for (auto& run : b->runs)
      if (run.geo == (int)g) {
        r = &run;
        break;
      }
    if (!G.fd || !G.Vt[0] || !r) continue;
    std::string key = "fdtc dim=" + std::to_string(r->dim) + " np=";
    for (int a = 0; a < r->dim; ++a) key += (a ? "," : "") + std::to_string(G.np[a]);
    key += " mixed dev=" + b->dev_name;
    std::vector<double> hit;
    if (tune_cache_get(key, hit) && hit.size() == 7 && hit[0] >= 0 && hit[0] <= 5) {
      G.tc_variant = (int)hit[0];
      for (int c = 0; c < 6; ++c) G.tc_ms[c] = (float)hit[1 + c];
      continue;
    }
    const C<float>* x = static_cast<const C<float>*>(b->w_p);
    C<float>* y = static_cast<C<float>*>(b->w_q);
    float* w[4] = {static_cast<float*>(b->w_qa), static_cast<float*>(b->w_qb), static_cast<float*>(b->w_qc),
                   static_cast<float*>(b->w_qd)};
    for (int c = 0; c < 6 && rc == TDZ_OK; ++c) {
      G.tc_variant = c;
      rc = fd_apply32(b, r, x, y, w[0], w[1], w[2], w[3], 0.025, nullptr);
      float tmin = 0.f;
      for (int k = 0; k < 3 && rc == TDZ_OK; ++k) {
        cudaEventRecord(e0, b->st);
        rc = fd_apply32(b, r, x, y, w[0], w[1], w[2], w[3], 0.025, nullptr);
        cudaEventRecord(e1, b->st);
        float ms = 0.f;
        if (rc == TDZ_OK &&
            (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
          rc = TDZ_ECUDA;
        tmin = k == 0 ? ms : std::min(tmin, ms);
      }
      G.tc_ms[c] = tmin;
    }
    int best = 0;
    for (int c = 1; c < 6; ++c)
      if (G.tc_ms[c] < G.tc_ms[best]) best = c;
    G.tc_variant = best;
    if (rc == TDZ_OK) {
      std::vector<double> vals{(double)best};
      for (int c = 0; c < 6; ++c) vals.push_back((double)G.tc_ms[c]);
      tune_cache_put(key, vals);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int werr = 0;  // a wait that ran out while timing
  if (rc == TDZ_OK && (cudaMemcpy(&werr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || werr != 0))
    rc = TDZ_ECUDA;
  return rc;
}

// z = M^-1 res and d_red[0..1] += res^T z (the rho of COCG; d_red zeroed by the caller): on the fast
// diagonalisation path the product is accumulated while the result is written
template <class T, int P>
void precond_dot(NdBatch* b, NdRun* r, Apply<T, P>& op, const C<T>* res, C<T>* z, double tau, double* dot) {
  if (use_fd(b, r)) {
    if constexpr (std::is_same<T, float>::value) {
      const int rc = fd_apply32(b, r, res, z, reinterpret_cast<float*>(op.qa), reinterpret_cast<float*>(op.qb),
                                static_cast<float*>(b->w_qc), static_cast<float*>(b->w_qd), tau, dot);
      if (rc != TDZ_OK && r->status == TDZ_OK) r->status = rc;
    } else {
      fd_apply64(b, r, res, z, reinterpret_cast<double*>(op.qa), reinterpret_cast<double*>(op.qb), tau, dot);
    }
    return;
  }
  cudaMemcpyAsync(z, res, sizeof(C<T>) * r->N, cudaMemcpyDeviceToDevice, b->st);
  line_precond<T, P>(b, r, z);
  k_bdot<T><<<grid_for(r->N), TPB, 0, b->st>>>(res, z, r->N, dot, b->gr);
}

// reads the reduction slots (and, in the same copy, the error word in the last slot)
double* red_get(NdBatch* b, int k, double* host) {
  double all[16];
  cudaMemcpyAsync(all, b->d_red, sizeof(all), cudaMemcpyDeviceToHost, b->st);
  cudaStreamSynchronize(b->st);
  for (int q = 0; q < k; ++q) host[q] = all[q];
  int werr = 0;
  std::memcpy(&werr, &all[15], sizeof(int));
  b->wait_failed = werr != 0;
  return host;
}

void red_zero(NdBatch* b, int k) { cudaMemsetAsync(b->d_red, 0, sizeof(double) * k, b->st); }

// Preconditioned COCG on A x = r (x starts at 0). Returns iterations; final ||r||^2 in *rr.
// The step lengths alpha = rho / (p^T q) and beta = rho_new / rho are formed on the device from the
// reduction slots (rho alternates between two slots, so no kernel reads a slot it overwrites), and
// the host reads the slots once per iteration, after the update, for the convergence test.
// Slots of d_red: [0..1] p^T q, [2] ||r||^2, [4..5] and [6..7] rho.
template <class T, int P>
int cocg(NdBatch* b, NdRun* r, Apply<T, P>& op, C<T>* x, C<T>* res, C<T>* z, C<T>* p, C<T>* q, double tau,
         const double* ebar, double tol_abs2, int maxit, double* rr_out) {
  const long long N = r->N;
  double h[8];
  double* const pq = b->d_red;
  double* const rrs = b->d_red + 2;
  double* rho_slot[2] = {b->d_red + 4, b->d_red + 6};
  int cur = 0;
  cudaMemsetAsync(x, 0, sizeof(C<T>) * N, b->st);
  red_zero(b, 8);
  precond_dot<T, P>(b, r, op, res, z, tau, rho_slot[cur]);
  cudaMemcpyAsync(p, z, sizeof(C<T>) * N, cudaMemcpyDeviceToDevice, b->st);
  k_nrm<T><<<grid_for(N), TPB, 0, b->st>>>(res, N, rrs, b->gr);
  double rr = red_get(b, 8, h)[2];
  int it = 0;
  if (b->wait_failed || (h[4] == 0.0 && h[5] == 0.0)) {
    *rr_out = rr;
    return 0;
  }
  while (rr > tol_abs2 && it < maxit) {
    op.apply(p, q, tau, ebar);
    cudaMemsetAsync(pq, 0, sizeof(double) * 3, b->st);
    k_bdot<T><<<grid_for(N), TPB, 0, b->st>>>(p, q, N, pq, b->gr);
    k_cocg_update_dev<T><<<grid_for(N), TPB, 0, b->st>>>(x, res, p, q, N, rho_slot[cur], pq, rrs, b->gr);
    red_get(b, 8, h);
    if (b->wait_failed || (h[0] == 0.0 && h[1] == 0.0)) break;  // p^T q = 0: the update was skipped
    rr = h[2];
    ++it;
    if (!(rr > tol_abs2)) break;
    const int nxt = 1 - cur;
    cudaMemsetAsync(rho_slot[nxt], 0, sizeof(double) * 2, b->st);
    precond_dot<T, P>(b, r, op, res, z, tau, rho_slot[nxt]);
    k_xpby_dev<T><<<grid_for(N), TPB, 0, b->st>>>(p, z, N, rho_slot[nxt], rho_slot[cur]);
    cur = nxt;
  }
  *rr_out = rr;
  return it;
}

// complex symmetric band LDL^T (host, binary64) of P_a = S_a + i tau mbar T1_a; upload in T
template <class T>
int factor_precond(NdBatch* b, NdRun* r, const tdz::Ops& o, double tau) {
  for (int ax = 0; ax < r->dim; ++ax) {
    const int n = r->n[ax], P = r->P, P1 = P + 1;
    std::vector<std::complex<double>> a((size_t)n * P1);
    for (size_t k = 0; k < a.size(); ++k) a[k] = {o.Sa[ax].a[k], tau * r->mbar * o.T1a[ax].a[k]};
    std::vector<std::complex<double>> L((size_t)n * P), Dv(n);
    std::vector<std::complex<double>> l(P1);
    for (int j = 0; j < n; ++j) {
      const std::complex<double> dj = a[(size_t)j * P1];
      const std::complex<double> di = 1.0 / dj;
      Dv[j] = di;
      const int rmax = std::min(P, n - 1 - j);
      for (int q = 1; q <= rmax; ++q) l[q] = a[(size_t)(j + q) * P1 + q] * di;
      for (int q = 1; q <= rmax; ++q) {
        for (int c = 1; c <= q; ++c) a[(size_t)(j + q) * P1 + (q - c)] -= l[q] * l[c] * dj;
        L[(size_t)j * P + q - 1] = l[q];
      }
    }
    std::vector<C<T>> hL(L.size()), hD(n);
    for (size_t k = 0; k < L.size(); ++k) hL[k] = C<T>{(T)L[k].real(), (T)L[k].imag()};
    for (int j = 0; j < n; ++j) hD[j] = C<T>{(T)Dv[j].real(), (T)Dv[j].imag()};
    cudaMemcpyAsync(b->pre_L[ax], hL.data(), sizeof(C<T>) * hL.size(), cudaMemcpyHostToDevice, b->st);
    cudaMemcpyAsync(b->pre_D[ax], hD.data(), sizeof(C<T>) * n, cudaMemcpyHostToDevice, b->st);
    cudaStreamSynchronize(b->st);
  }
  return TDZ_OK;
}

inline ff ff_of(double v) {
  const float h = (float)v;
  return ff{h, (float)(v - (double)h)};
}
MediumFF medium_ff(const MediumDev& d) {
  MediumFF m{};
  m.mass_kind = d.mass_kind;
  m.pot_kind = d.pot_kind;
  m.m0 = ff_of(1.0 / d.mp[0]);
  if (d.mass_kind == TDZ_MASS_ELLIPSE) {
    m.ia = ff_of(1.0 / d.mp[0]);
    m.ib = ff_of(1.0 / d.mp[1]);
    m.min_ = ff_of(1.0 / d.mp[2]);
    m.mout = ff_of(1.0 / d.mp[3]);
  }
  m.z = ff_of(d.vp[0]);
  m.eps = ff_of(d.vp[1]);
  for (int a = 0; a < 3; ++a) m.w2[a] = ff_of(d.vp[a] * d.vp[a]);
  return m;
}

// observables of the state c (given in the operator's arithmetic T: binary64 or double-float):
// [d_a, a_a, norm]; y is scratch of the state's size
// The observables of a state row (Sec. "Dipoles"): out[a] = c^H D_a c, out[D + a] = the acceleration
// -c^H G_a c - E_a(t) c^H K c (Eq. pdm_acceleration), out[2D] = c^H S c. observe_kron forms the
// Kronecker-product ones (norm, dipoles), observe_quad the Gauss-point ones (G_a, and K with a
// variable mass), observe_finish the accelerations from them.
template <class T, int P>
void observe_kron(NdBatch* b, NdRun* r, Apply<T, P>& op, const C<T>* c, C<T>* y, double* out) {
  const long long N = r->N;
  double h[4];
  double zero3[3] = {0, 0, 0};
  double norm = 0.0, dvals[3] = {0, 0, 0};
  if (r->dim == 2) {
    // x-passes t = S_x c, u = D_x c, then the three forms in one y-pass
    const AxisDev& A0 = r->ax[0];
    BandTerms<T> bs{}, bd{};
    bs.nt = bd.nt = 1;
    bs.R[0] = tab<T>(A0, TS);
    bd.R[0] = tab<T>(A0, TD);
    bs.cr[0] = bd.cr[0] = 1;
    const long long tot = N;
    launch_axis_band<T, P>(b->st, grid_for(tot), bs, c, c, op.t1, r->n[1], r->n[0], 1);
    launch_axis_band<T, P>(b->st, grid_for(tot), bd, c, c, op.t2, r->n[1], r->n[0], 1);
    red_zero(b, 3);
    k_qform2_y<T, P><<<grid_for(N), TPB, 0, b->st>>>(c, op.t1, op.t2, tab<T>(r->ax[1], TS), tab<T>(r->ax[1], TD),
                                                     r->n[0], r->n[1], b->d_red, b->gr);
    double q3[3];
    red_get(b, 3, q3);
    norm = q3[0];
    dvals[0] = q3[1];
    dvals[1] = q3[2];
  } else {
    op.kron(c, y, 1, 0.0, zero3);
    red_zero(b, 2);
    k_hdot<T><<<grid_for(N), TPB, 0, b->st>>>(c, y, N, b->d_red, b->gr);
    norm = red_get(b, 2, h)[0];
    for (int a = 0; a < r->dim; ++a) {
      op.kron(c, y, 2, 0.0, zero3, a);
      red_zero(b, 2);
      k_hdot<T><<<grid_for(N), TPB, 0, b->st>>>(c, y, N, b->d_red, b->gr);
      dvals[a] = red_get(b, 2, h)[0];
    }
  }
  for (int a = 0; a < r->dim; ++a) out[a] = dvals[a];
  out[2 * r->dim] = norm;
}
// q4[a] = c^H G_a c (a < dim), q4[3] = c^H K c (variable mass), by one double-float Gauss-point pass
template <class T, int P>
void observe_quad(NdBatch* b, NdRun* r, Apply<T, P>& op, const C<T>* c, double* q4) {
  const C<T>* X = op.to_pencils(c, -1);
  const int L = r->dim - 1;
  long long inner = 1;
  for (int a = 0; a < L; ++a) inner *= r->Q[a];
  const AxisDev& AL = r->ax[L];
  int echunk = 1;
  const long long nch = reduce_nchunks(AL.E, inner, P, &echunk);
  red_zero(b, 4);
  k_fused_last_reduce_ff<P, T><<<grid_for(inner * nch), TPB, 0, b->st>>>(X, r->ax[0], r->ax[1], AL, r->dim, inner,
                                                                         echunk, medium_ff(r->med),
                                                                         r->const_mass ? 0 : 1, b->geo[r->geo].Gq,
                                                                         b->d_red, b->gr);
  red_get(b, 4, q4);
}
void observe_finish(const NdRun* r, const double* q4, const double* Et, double* out) {
  const int D = r->dim;
  const double kq = r->const_mass ? r->cm * out[2 * D] : q4[3];
  for (int a = 0; a < D; ++a) out[D + a] = -q4[a] - Et[a] * kq;
}
template <class T, int P>
void observe(NdBatch* b, NdRun* r, Apply<T, P>& op, const C<T>* c, C<T>* y, const double* Et, double* out) {
  double q4[4];
  observe_kron<T, P>(b, r, op, c, y, out);
  observe_quad<T, P>(b, r, op, c, q4);
  observe_finish(r, q4, Et, out);
}

template <int P>
int propagate_run(NdBatch* b, NdRun* r, const tdz::Ops& o, const double* field, double dt, long long step0,
                  long long nsteps, double* obs_out) {
  const long long N = r->N;
  const double tau = 0.5 * dt;
  const int D = r->dim;
  const bool mixed = b->prec == TDZ_MIXED;
  const NdGeo& G = b->geo[r->geo];
  const bool stencil = G.has_stencil() && b->opt_operator != TDZ_OPERATOR_QUADRATURE;
  if (!use_fd(b, r)) {
    if (mixed) factor_precond<float>(b, r, o, tau);
    else factor_precond<double>(b, r, o, tau);
  }
  C<double>* c = reinterpret_cast<C<double>*>(r->c);
  double h[4];
  if (!mixed) {
    // binary64 throughout: r0 = 2 (S c - A c), COCG on A delta = r0 to the tolerance, c += delta
    Apply<double, P> op{b, r, reinterpret_cast<C<double>*>(b->d_t1), reinterpret_cast<C<double>*>(b->d_t2),
                        reinterpret_cast<C<double>*>(b->d_t3), reinterpret_cast<C<double>*>(b->d_t4),
                        reinterpret_cast<C<double>*>(b->d_qa), reinterpret_cast<C<double>*>(b->d_qb)};
    if (stencil) op.Wm = G.W64;
    C<double>* r0 = reinterpret_cast<C<double>*>(b->d_r0);
    C<double>* y = reinterpret_cast<C<double>*>(b->d_y);
    for (long long s = 0; s < nsteps && r->status == TDZ_OK; ++s) {
      double ebar[3] = {0, 0, 0}, Et[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) {
        ebar[a] = 0.5 * (field[s * D + a] + field[(s + 1) * D + a]);
        Et[a] = field[(s + 1) * D + a];
      }
      double zero3[3] = {0, 0, 0};
      op.apply(c, y, tau, ebar);
      op.kron(c, r0, 1, 0.0, zero3);
      red_zero(b, 1);
      k_nrm<double><<<grid_for(N), TPB, 0, b->st>>>(r0, N, b->d_red, b->gr);
      const double bb = red_get(b, 1, h)[0];
      k_axby<double, double><<<grid_for(N), TPB, 0, b->st>>>(y, r0, N, -2.0, 2.0);
      double rr = 0;
      const int its = cocg<double, P>(b, r, op, y, r0, reinterpret_cast<C<double>*>(b->d_z),
                                      reinterpret_cast<C<double>*>(b->d_p), reinterpret_cast<C<double>*>(b->d_q), tau,
                                      ebar, b->tol * b->tol * bb, b->max_it, &rr);
      r->iters += its;
      r->nsolve++;
      const double rel = std::sqrt(rr / std::max(bb, 1e-300));
      k_axby<double, double><<<grid_for(N), TPB, 0, b->st>>>(y, c, N, 1.0, 1.0);  // c += delta
      r->max_rel = std::max(r->max_rel, rel);
      if (!(rel <= b->tol) && r->status == TDZ_OK) r->status = TDZ_ENOCONV;
      double* row = obs_out + s * (2 + 3 * D);
      row[0] = (double)(step0 + s + 1) * dt;
      for (int a = 0; a < D; ++a) row[1 + a] = Et[a];
      observe<double, P>(b, r, op, c, y, Et, row + 1 + D);
      if (!std::isfinite(row[1 + 3 * D]) || !std::isfinite(row[1 + D])) r->status = TDZ_ENONFINITE;
    }
  } else {
    // mixed: the binary64-class residuals r0 = 2 (S c - A c) and r = r0 - A delta in double-float,
    // inner solves by FP32 COCG, delta accumulated in double-float, c += delta in binary64
    Apply<fx, P> opx{b, r, reinterpret_cast<C<fx>*>(b->d_t1), reinterpret_cast<C<fx>*>(b->d_t2),
                     reinterpret_cast<C<fx>*>(b->d_t3), reinterpret_cast<C<fx>*>(b->d_t4),
                     reinterpret_cast<C<fx>*>(b->d_qa), reinterpret_cast<C<fx>*>(b->d_qb)};
    Apply<float, P> op32{b, r, static_cast<C<float>*>(b->w_t1), static_cast<C<float>*>(b->w_t2),
                         static_cast<C<float>*>(b->w_t3), static_cast<C<float>*>(b->w_t4),
                         static_cast<C<float>*>(b->w_qa), static_cast<C<float>*>(b->w_qb)};
    if (stencil) {
      opx.Wm = G.Wx;
      // the FP32 stencil is stored tile-major for the fused apply, which has no absorbing-layer term; with
      // a layer the FP32 inner solve applies V and the mass term by quadrature instead (the same operator)
      op32.Wm = r->cap ? nullptr : G.W32;
    }
    opx.Vtab = G.Vqx;  // the FP32 inner solve evaluates the potential at the points instead
    C<fx>* cx_ = reinterpret_cast<C<fx>*>(b->d_z);    // c in double-float
    C<fx>* r0 = reinterpret_cast<C<fx>*>(b->d_r0);
    C<fx>* y = reinterpret_cast<C<fx>*>(b->d_y);      // A c, then delta
    C<fx>* rc = reinterpret_cast<C<fx>*>(b->d_rc);    // current residual
    C<float>* rf = static_cast<C<float>*>(b->w_r);
    C<float>* xf = static_cast<C<float>*>(b->w_x);
    // Where the residual apply runs the double-float potential pass at the Gauss points (quadrature
    // operator, soft-core point factor tabulated, constant mass), the Gauss-point observables of a step's
    // new state are reduced inside the next step's first residual apply, whose input is that state: the
    // row stays open until then (the last row of the call is closed by the standalone pass).
    const bool defer_obs = !stencil && r->const_mass && r->med.pot_kind == TDZ_POT_SOFTCORE && G.Gq != nullptr;
    double* open_row = nullptr;  // the row whose c^H G_a c is pending (reduction slots 8..10)
    auto close_row = [&](const double* g3) {
      double q4[4] = {g3[0], g3[1], g3[2], 0.0};
      observe_finish(r, q4, open_row + 1, open_row + 1 + D);
      open_row = nullptr;
    };
    for (long long s = 0; s < nsteps && r->status == TDZ_OK && !b->wait_failed; ++s) {
      double ebar[3] = {0, 0, 0}, Et[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) {
        ebar[a] = 0.5 * (field[s * D + a] + field[(s + 1) * D + a]);
        Et[a] = field[(s + 1) * D + a];
      }
      double zero3[3] = {0, 0, 0};
      k_axby<double, fx><<<grid_for(N), TPB, 0, b->st>>>(c, cx_, N, 1.0, 0.0);
      if (open_row) {
        cudaMemsetAsync(b->d_red + 8, 0, sizeof(double) * 3, b->st);
        opx.obs_gtab = G.Gq;
        opx.obs_res = b->d_red + 8;
      }
      opx.apply(cx_, y, tau, ebar);
      opx.kron(cx_, r0, 1, 0.0, zero3);
      red_zero(b, 1);
      k_nrm<fx><<<grid_for(N), TPB, 0, b->st>>>(r0, N, b->d_red, b->gr);
      double h16[16];
      const double bb = red_get(b, 16, h16)[0];
      if (open_row) close_row(h16 + 8);
      const double tol2 = b->tol * b->tol * bb;
      k_axby<fx, fx><<<grid_for(N), TPB, 0, b->st>>>(y, r0, N, -2.0, 2.0);
      cudaMemsetAsync(y, 0, sizeof(C<fx>) * N, b->st);  // y is delta from here on
      cudaMemcpyAsync(rc, r0, sizeof(C<fx>) * N, cudaMemcpyDeviceToDevice, b->st);
      double rr = bb * 1e300;
      red_zero(b, 1);
      k_nrm<fx><<<grid_for(N), TPB, 0, b->st>>>(rc, N, b->d_red, b->gr);
      rr = red_get(b, 1, h)[0];
      // Each FP32 solve contracts the residual by a factor rho, measured on the first one; when the
      // next solve is predicted to end at or below a tenth of the tolerance (and rho < 1e-2), its
      // residual is not formed (one double-float apply saved), the same rule as the 1-D path.
      double rho = 1.0;
      for (int outer = 0; outer < 8 && rr > tol2 && !b->wait_failed; ++outer) {
        k_axby<fx, float><<<grid_for(N), TPB, 0, b->st>>>(rc, rf, N, 1.0, 0.0);
        double rri = 0;
        const int its = cocg<float, P>(b, r, op32, xf, rf, static_cast<C<float>*>(b->w_z),
                                       static_cast<C<float>*>(b->w_p), static_cast<C<float>*>(b->w_q), tau, ebar,
                                       rr * b->inner_tol * b->inner_tol, b->max_it, &rri);
        r->iters += its;
        r->nsolve++;
        k_axby<float, fx><<<grid_for(N), TPB, 0, b->st>>>(xf, y, N, 1.0, 1.0);
        const double predicted2 = rho * rho * rr;
        if (outer >= 1 && rho < 1e-2 && predicted2 <= 0.01 * tol2) {
          rr = predicted2;  // accepted unchecked
          break;
        }
        opx.apply(y, rc, tau, ebar);                                         // rc = A delta
        k_axby<fx, fx><<<grid_for(N), TPB, 0, b->st>>>(r0, rc, N, 1.0, -1.0);  // rc = r0 - A delta
        red_zero(b, 1);
        k_nrm<fx><<<grid_for(N), TPB, 0, b->st>>>(rc, N, b->d_red, b->gr);
        const double rr_new = red_get(b, 1, h)[0];
        if (outer == 0) rho = std::min(1.0, std::sqrt(rr_new / std::max(rr, 1e-300)));
        rr = rr_new;
      }
      const double rel = std::sqrt(rr / std::max(bb, 1e-300));
      k_axby<fx, double><<<grid_for(N), TPB, 0, b->st>>>(y, c, N, 1.0, 1.0);  // c += delta
      r->max_rel = std::max(r->max_rel, rel);
      if (!(rel <= b->tol) && r->status == TDZ_OK) r->status = TDZ_ENOCONV;
      double* row = obs_out + s * (2 + 3 * D);
      row[0] = (double)(step0 + s + 1) * dt;
      for (int a = 0; a < D; ++a) row[1 + a] = Et[a];
      k_axby<double, fx><<<grid_for(N), TPB, 0, b->st>>>(c, cx_, N, 1.0, 0.0);
      if (defer_obs) {
        observe_kron<fx, P>(b, r, opx, cx_, y, row + 1 + D);
        open_row = row;
      } else {
        observe<fx, P>(b, r, opx, cx_, y, Et, row + 1 + D);
      }
      if (!std::isfinite(row[1 + 3 * D]) || !std::isfinite(row[1 + D])) r->status = TDZ_ENONFINITE;
    }
    if (open_row) {  // cx_ still holds the last step's state
      double q4[4];
      observe_quad<fx, P>(b, r, opx, cx_, q4);
      close_row(q4);
    }
  }
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return nd_cuda_fail(e, "tdz_propagate (2-D/3-D)");
  int werr = 0;
  e = cudaMemcpy(&werr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return nd_cuda_fail(e, "tdz_propagate (2-D/3-D)");
  if (werr != 0) {
    cudaMemsetAsync(b->d_err, 0, sizeof(int), b->st);
    cudaStreamSynchronize(b->st);
    b->wait_failed = false;
    r->status = TDZ_ECUDA;
    set_error("tdz_propagate (2-D): a stencil tile copy did not complete within the wait limit");
    return TDZ_ECUDA;
  }
  return TDZ_OK;
}

// Ground state of H0 c = eps S c (Eq. gen_ev) for one 2-D/3-D run, by inverse iteration with a fixed
// shift sigma below the spectrum: x = (H0 - sigma S)^-1 S c solved by the batch's preconditioned COCG on
// i tau (H0 - sigma S) (the operator A - (1 + i tau sigma) S, tau = 1, no field, fast-diagonalisation
// preconditioner with the shifted eigenvalue scaling), then eps = sigma + c^H S x / x^H S x (the
// Rayleigh quotient of x, since (H0 - sigma S) x = S c) and c <- x / |x|_S. It stops when the
// eigen-residual |H0 c - eps S c|_{S^-1}, formed from the solve as S (c_old / |x|_S - (eps - sigma) c_new),
// is at most tol |eps|. T = double in a binary64 batch; T = float in a mixed batch (the FP32 operator and
// preconditioner of its inner solves, residuals to FP32 accuracy). The run's state is the start vector
// and is replaced by the result (S-normalised).
template <class T, int P>
int ground_state_run(NdBatch* b, NdRun* r, double sigma, double tol, int max_outer, double* energy, int* outer_out,
                     double* resid_out) {
  const long long N = r->N;
  const double tau = 1.0;
  double zero3[3] = {0, 0, 0};
  const bool f32 = std::is_same<T, float>::value;
  const NdGeo& G = b->geo[r->geo];
  const bool stencil = G.has_stencil() && b->opt_operator != TDZ_OPERATOR_QUADRATURE;
  auto vec = [&](void* d64, void* w32) { return static_cast<C<T>*>(f32 ? w32 : d64); };
  Apply<T, P> op{b, r, vec(b->d_t1, b->w_t1), vec(b->d_t2, b->w_t2), vec(b->d_t3, b->w_t3), vec(b->d_t4, b->w_t4),
                 vec(b->d_qa, b->w_qa), vec(b->d_qb, b->w_qb)};
  if (stencil) {
    if constexpr (std::is_same<T, float>::value) op.Wm = G.W32;
    else op.Wm = G.W64;
  }
  // binary64: the run state itself, then the propagator's binary64 work vectors; FP32: the iterate in the
  // (unused) binary64 residual buffer, the FP32 solve's vectors; S products in d_rc either way
  C<double>* c64 = reinterpret_cast<C<double>*>(r->c);
  C<T>* c = f32 ? reinterpret_cast<C<T>*>(b->d_r0) : reinterpret_cast<C<T>*>(r->c);
  C<T>* rhs = f32 ? static_cast<C<T>*>(b->w_r) : reinterpret_cast<C<T>*>(b->d_r0);
  C<T>* x = vec(b->d_y, b->w_x);
  C<T>* s = reinterpret_cast<C<T>*>(b->d_rc);
  C<T>* z = vec(b->d_z, b->w_z);
  C<T>* pp = vec(b->d_p, b->w_p);
  C<T>* qq = vec(b->d_q, b->w_q);
  double h[16];
  auto hdot = [&](const C<T>* u, const C<T>* v) {
    red_zero(b, 2);
    k_hdot<T><<<grid_for(N), TPB, 0, b->st>>>(u, v, N, b->d_red, b->gr);
    return red_get(b, 2, h)[0];
  };
  if (f32) k_axby<double, T><<<grid_for(N), TPB, 0, b->st>>>(c64, c, N, 1.0, 0.0);
  b->eig = true;
  b->eig_sigma = sigma;
  int rc = TDZ_ENOCONV, k = 0;
  double eps = 0.0, rel = 1e300;
  op.kron(c, rhs, 1, 0.0, zero3);  // S-normalise the start vector
  const double n0 = hdot(c, rhs);
  if (!(n0 > 0.0) || !std::isfinite(n0)) {
    b->eig = false;
    set_error("tdz_batch_ground_state: the start vector has no S-norm");
    return TDZ_EINVAL;
  }
  k_caxpby<T><<<grid_for(N), TPB, 0, b->st>>>(c, c, N, 1.0 / std::sqrt(n0), 0.0, 0.0, 0.0);
  for (k = 1; k <= max_outer && !b->wait_failed; ++k) {
    op.kron(c, rhs, 1, 0.0, zero3);                                                    // S c
    k_caxpby<T><<<grid_for(N), TPB, 0, b->st>>>(rhs, rhs, N, 0.0, tau, 0.0, 0.0);      // i tau S c
    red_zero(b, 1);
    k_nrm<T><<<grid_for(N), TPB, 0, b->st>>>(rhs, N, b->d_red, b->gr);
    const double bb = red_get(b, 1, h)[0];
    double rr = 0.0;
    const double tin = std::max(0.1 * tol, f32 ? 1e-6 : 1e-13);
    const int its = cocg<T, P>(b, r, op, x, rhs, z, pp, qq, tau, zero3, tin * tin * bb, b->max_it, &rr);
    r->iters += its;
    r->nsolve++;
    op.kron(x, s, 1, 0.0, zero3);  // S x
    const double xsx = hdot(x, s), csx = hdot(c, s);
    if (!(xsx > 0.0) || !std::isfinite(xsx)) {
      rc = TDZ_ENONFINITE;
      break;
    }
    eps = sigma + csx / xsx;
    const double ix = 1.0 / std::sqrt(xsx);
    // w = c_old / |x|_S - (eps - sigma) x / |x|_S in rhs, then |w|_S
    cudaMemcpyAsync(rhs, c, sizeof(C<T>) * N, cudaMemcpyDeviceToDevice, b->st);
    k_caxpby<T><<<grid_for(N), TPB, 0, b->st>>>(x, rhs, N, -(eps - sigma) * ix, 0.0, ix, 0.0);
    op.kron(rhs, s, 1, 0.0, zero3);
    const double ww = hdot(rhs, s);
    k_caxpby<T><<<grid_for(N), TPB, 0, b->st>>>(x, c, N, ix, 0.0, 0.0, 0.0);  // c = x / |x|_S
    rel = std::sqrt(std::max(ww, 0.0)) / std::max(std::fabs(eps), 1e-300);
    if (rel <= tol) {
      rc = TDZ_OK;
      break;
    }
  }
  b->eig = false;
  if (f32) k_axby<T, double><<<grid_for(N), TPB, 0, b->st>>>(c, c64, N, 1.0, 0.0);
  if (b->wait_failed) rc = TDZ_ECUDA;
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return nd_cuda_fail(e, "tdz_batch_ground_state");
  if (energy) *energy = eps;
  if (outer_out) *outer_out = std::min(k, max_outer);
  if (resid_out) *resid_out = rel;
  if (rc == TDZ_ENOCONV) set_error("tdz_batch_ground_state: the eigen-residual did not reach the tolerance");
  return rc;
}

// work buffers of one worker, sized for the largest run of the batch (maxN, maxQ, maxSide, maxn set)
bool alloc_work(NdBatch* b) {
  const size_t z64 = sizeof(double2), maxN = b->maxN, maxQ = b->maxQ;
  bool ok = true;
  b->d_r0 = static_cast<double2*>(b->alloc(z64 * maxN));
  b->d_y = static_cast<double2*>(b->alloc(z64 * maxN));
  b->d_t1 = static_cast<double2*>(b->alloc(z64 * maxN));
  b->d_t2 = static_cast<double2*>(b->alloc(z64 * maxN));
  b->d_t3 = static_cast<double2*>(b->alloc(z64 * maxN));
  b->d_t4 = static_cast<double2*>(b->alloc(z64 * maxN));
  b->d_qa = static_cast<double2*>(b->alloc(z64 * maxQ));
  b->d_qb = static_cast<double2*>(b->alloc(z64 * maxQ));
  b->d_red = static_cast<double*>(b->alloc(sizeof(double) * 16));
  b->gr.part = static_cast<double*>(b->alloc(sizeof(double) * 4 * 148 * 16));  // grid_for's block cap
  b->gr.ticket = static_cast<unsigned*>(b->alloc(sizeof(unsigned) * 4));
  ok = ok && b->gr.part && b->gr.ticket;
  b->d_err = b->d_red ? reinterpret_cast<int*>(b->d_red + 15) : nullptr;  // red_zero never clears it
  if (b->prec == TDZ_MIXED && b->dim == 2)
    for (int a = 0; a < 2; ++a) {
      b->rb32[a] = static_cast<float2*>(b->alloc(sizeof(float2) * (size_t)std::max(b->maxn, 1) * (2 * b->P + 2)));
      ok = ok && b->rb32[a];
    }
  b->d_side = b->alloc(sizeof(double2) * std::max<size_t>(b->maxSide, 1));
  b->d_z = static_cast<double2*>(b->alloc(z64 * maxN));
  b->d_p = static_cast<double2*>(b->alloc(z64 * maxN));
  b->d_q = static_cast<double2*>(b->alloc(z64 * maxN));
  b->d_rc = static_cast<double2*>(b->alloc(z64 * maxN));
  ok = ok && b->d_r0 && b->d_y && b->d_t1 && b->d_t2 && b->d_t3 && b->d_t4 && b->d_qa && b->d_qb && b->d_red &&
            b->d_side && b->d_z && b->d_p && b->d_q && b->d_rc;
  const size_t zs = b->prec == TDZ_MIXED ? sizeof(float2) : sizeof(double2);
  for (int a = 0; a < 3; ++a) {
    b->pre_L[a] = b->alloc(zs * (size_t)std::max(b->maxn, 1) * b->P);
    b->pre_D[a] = b->alloc(zs * (size_t)std::max(b->maxn, 1));
    ok = ok && b->pre_L[a] && b->pre_D[a];
  }
  if (b->prec == TDZ_MIXED) {
    const size_t f = sizeof(float2);
    void** w[] = {&b->w_x, &b->w_r, &b->w_z, &b->w_p, &b->w_q, &b->w_t1, &b->w_t2, &b->w_t3, &b->w_t4};
    for (void** pp : w) {
      *pp = b->alloc(f * maxN);
      ok = ok && *pp;
    }
    b->w_qa = b->alloc(f * maxQ);
    b->w_qb = b->alloc(f * maxQ);
    b->w_qc = b->alloc(f * std::max<size_t>(b->maxPad, 1));
    b->w_qd = b->alloc(f * std::max<size_t>(b->maxPad, 1));
    ok = ok && b->w_qa && b->w_qb && b->w_qc && b->w_qd;
  }
  return ok;
}

// Extra workers for a batch of several runs (up to 8, within a quarter of the free device memory)
int make_workers(NdBatch* b) {
  // host threads (one stream each) that propagate runs concurrently: TDZ_ND_WORKERS (1..64), default 8
  int nmax = 8;
  if (const char* env = std::getenv("TDZ_ND_WORKERS")) {
    const int v = std::atoi(env);
    if (v >= 1 && v <= 64) nmax = v;
  }
  const int want = std::min(b->nruns, nmax) - 1;
  if (want <= 0) return TDZ_OK;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const size_t per = b->work_bytes;
  for (int k = 0; k < want && (size_t)(k + 1) * per < free_b / 4; ++k) {
    NdBatch* w = new (std::nothrow) NdBatch;
    if (!w) return TDZ_ENOMEM;
    w->prec = b->prec;
    w->dim = b->dim;
    w->P = b->P;
    w->nruns = 0;
    w->geo = b->geo;
    w->maxN = b->maxN;
    w->maxQ = b->maxQ;
    w->maxPad = b->maxPad;
    w->maxSide = b->maxSide;
    w->maxn = b->maxn;
    w->nsm = b->nsm;
    if (cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete w;
      return TDZ_ECUDA;
    }
    w->own_stream = true;
    if (cublasCreate(&w->blas) != CUBLAS_STATUS_SUCCESS || cublasSetStream(w->blas, w->st) != CUBLAS_STATUS_SUCCESS) {
      delete w;
      return TDZ_ECUDA;
    }
    if (!alloc_work(w)) {
      delete w;
      return TDZ_ENOMEM;
    }
    if (cudaStreamSynchronize(w->st) != cudaSuccess) {
      delete w;
      return TDZ_ECUDA;
    }
    b->workers.push_back(w);
  }
  return TDZ_OK;
}

MediumDev medium_dev(const Medium& m) {
  MediumDev d{};
  d.mass_kind = m.mass_kind;
  d.pot_kind = m.pot_kind;
  std::memcpy(d.mp, m.mass_par, sizeof(d.mp));
  std::memcpy(d.vp, m.pot_par, sizeof(d.vp));
  return d;
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ f, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    f[i] = (float)a[i];
}

// V (np x np, V[k + j np] = component k of eigenvector j) rounded to TF32: Vt[j np + k] = V[k + j np]
// and its transpose VtT[j np + k] = V[j + k np] (the same rounded values)
__global__ void k_v_tf32(const double* __restrict__ V, float* __restrict__ Vt, float* __restrict__ VtT, int np) {
  const long long n = (long long)np * np;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long j = i / np, k = i - j * np;
    Vt[i] = tf32_hi((float)V[i]);
    VtT[i] = tf32_hi((float)V[k * np + j]);
  }
}

// Generalised symmetric eigenproblems T1_a v = lam S_a v of every axis (cuSOLVER, binary64), eigenvectors
// S_a-orthonormal. On a solver failure the geometry keeps the line preconditioner (fd = false).
int fd_setup(NdBatch* b, int g, const Ops& o) {
  NdGeo& G = b->geo[g];
  {
    // the split, scaling and merge kernels index a padded plane in 32 bits
    long long planes = 1;
    for (int a = 0; a < o.dim; ++a) planes *= (o.n[a] + 7) / 8 * 8;
    if (planes >= (1LL << 31)) return TDZ_OK;  // fd stays false: the line preconditioner is used
  }
  cusolverDnHandle_t h = nullptr;
  if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) return TDZ_OK;
  cusolverDnSetStream(h, b->st);
  bool ok = true;
  for (int a = 0; a < o.dim && ok; ++a) {
    const int n = (int)o.n[a], P = o.p[a];
    G.n[a] = n;
    std::vector<double> A((size_t)n * n, 0.0), B((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int d = 0; d <= P && d <= i; ++d) {
        const int j = i - d;
        A[(size_t)i + (size_t)j * n] = A[(size_t)j + (size_t)i * n] = o.T1a[a].at(i, d);
        B[(size_t)i + (size_t)j * n] = B[(size_t)j + (size_t)i * n] = o.Sa[a].at(i, d);
      }
    // factors stored zero-padded to np = n rounded up to 8 (np x np, eigenvalues padded with 0)
    const int np = (n + 7) / 8 * 8;
    G.np[a] = np;
    const bool mixed = b->prec == TDZ_MIXED;
    G.V64[a] = static_cast<double*>(b->alloc(sizeof(double) * np * np));
    if (mixed) {
      G.Vt[a] = static_cast<float*>(b->alloc(sizeof(float) * np * np));
      G.VtT[a] = static_cast<float*>(b->alloc(sizeof(float) * np * np));
      G.lam32[a] = static_cast<float*>(b->alloc(sizeof(float) * np));
    }
    G.lam[a] = static_cast<double*>(b->alloc(sizeof(double) * np));
    if (!G.V64[a] || !G.lam[a] || (mixed && (!G.Vt[a] || !G.VtT[a] || !G.lam32[a]))) {
      cusolverDnDestroy(h);
      return TDZ_ENOMEM;
    }
    double *dA = nullptr, *dB = nullptr;
    int* dinfo = nullptr;
    double* work = nullptr;
    int lwork = 0, info = -1;
    ok = cudaMalloc(&dA, sizeof(double) * A.size()) == cudaSuccess &&
         cudaMalloc(&dB, sizeof(double) * B.size()) == cudaSuccess && cudaMalloc(&dinfo, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(dA, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice, b->st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(dB, B.data(), sizeof(double) * B.size(), cudaMemcpyHostToDevice, b->st) == cudaSuccess;
    ok = ok && cusolverDnDsygvd_bufferSize(h, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                           dA, n, dB, n, G.lam[a], &lwork) == CUSOLVER_STATUS_SUCCESS;
    ok = ok && cudaMalloc(&work, sizeof(double) * std::max(lwork, 1)) == cudaSuccess;
    ok = ok && cusolverDnDsygvd(h, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, dA, n,
                                dB, n, G.lam[a], work, lwork, dinfo) == CUSOLVER_STATUS_SUCCESS;
    ok = ok && cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, b->st) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(b->st) == cudaSuccess && info == 0;
    ok = ok && cudaMemcpy2DAsync(G.V64[a], sizeof(double) * np, dA, sizeof(double) * n, sizeof(double) * n, n,
                                 cudaMemcpyDeviceToDevice, b->st) == cudaSuccess;
    if (ok && mixed) {
      k_v_tf32<<<grid_for((long long)np * np), TPB, 0, b->st>>>(G.V64[a], G.Vt[a], G.VtT[a], np);
      k_to_f32<<<grid_for(np), TPB, 0, b->st>>>(G.lam[a], G.lam32[a], np);
      ok = cudaStreamSynchronize(b->st) == cudaSuccess;
    }
    cudaFree(work);
    cudaFree(dinfo);
    cudaFree(dB);
    cudaFree(dA);
  }
  cusolverDnDestroy(h);
  G.fd = ok;
  return TDZ_OK;
}

template <int P>
int stencil_setup_p(NdBatch* b, NdGeo& G, const AxisDev& ax, const AxisDev& ay, const MediumDev& M, bool varmass) {
  constexpr int W = 2 * P + 1;
  const long long N = (long long)ax.n * ay.n;
  const size_t nf = (size_t)ay.Q * ax.n * W;
  const size_t nt = (size_t)ax.Q * ay.Q;
  const size_t nh = (size_t)N * half_count(P);
  if (b->prec == TDZ_MIXED) {
    const size_t ntiles = (size_t)ay.n * wt_tiles_per_row(ax.n);
    G.W32 = static_cast<float*>(b->alloc(sizeof(float) * ntiles * kWtRows * W * W));  // zero padded rows
    G.Wx = static_cast<fx*>(b->alloc(sizeof(fx) * nh));
    if (!G.W32 || !G.Wx) return TDZ_ENOMEM;
  } else {
    G.W64 = static_cast<double*>(b->alloc(sizeof(double) * nh));
    if (!G.W64) return TDZ_ENOMEM;
  }
  double *F1 = nullptr, *F2 = nullptr, *fV = nullptr, *fK = nullptr;
  if (cudaMalloc(&F1, sizeof(double) * nf) != cudaSuccess || cudaMalloc(&fV, sizeof(double) * nt) != cudaSuccess ||
      (varmass && (cudaMalloc(&F2, sizeof(double) * nf) != cudaSuccess ||
                   cudaMalloc(&fK, sizeof(double) * nt) != cudaSuccess))) {
    cudaFree(F1);
    cudaFree(F2);
    cudaFree(fV);
    cudaFree(fK);
    set_error("tdz_batch_create: no device memory for the 2-D stencil assembly");
    return TDZ_ENOMEM;
  }
  const int vm = varmass ? 1 : 0;
  k_w_ftab<<<grid_for((long long)nt), TPB, 0, b->st>>>(ax, ay, medium_t<double>(M), vm, fV, fK);
  k_w_stage1<P><<<grid_for((long long)ay.Q * ax.n), TPB, 0, b->st>>>(ax, ay, vm, fV, fK, F1, F2);
  k_w_stage2<P><<<grid_for(N * W), TPB, 0, b->st>>>(ax, ay, vm, F1, F2, G.W64, G.W32, G.Wx);
  cudaError_t e = cudaStreamSynchronize(b->st);
  cudaFree(F1);
  cudaFree(F2);
  cudaFree(fV);
  cudaFree(fK);
  if (e != cudaSuccess) return nd_cuda_fail(e, "tdz_batch_create (2-D stencil)");
  return TDZ_OK;
}

int stencil_setup(NdBatch* b, int g, const AxisDev& ax, const AxisDev& ay, const MediumDev& M, bool varmass) {
  NdGeo& G = b->geo[g];
  switch (b->P) {
    case 1: return stencil_setup_p<1>(b, G, ax, ay, M, varmass);
    case 2: return stencil_setup_p<2>(b, G, ax, ay, M, varmass);
    case 3: return stencil_setup_p<3>(b, G, ax, ay, M, varmass);
    case 4: return stencil_setup_p<4>(b, G, ax, ay, M, varmass);
    case 5: return stencil_setup_p<5>(b, G, ax, ay, M, varmass);
    case 6: return stencil_setup_p<6>(b, G, ax, ay, M, varmass);
    case 7: return stencil_setup_p<7>(b, G, ax, ay, M, varmass);
    default: return stencil_setup_p<8>(b, G, ax, ay, M, varmass);
  }
}

}  // namespace

namespace tdz {

int nd_batch_create(const tdz_ops* const* ops, int nops, int nruns, const int* ops_index, int precision, void* stream,
                    NdBatch** out) {
  const int dim = ops[0]->o.dim;
  const int P = ops[0]->o.p[0];
  for (int g = 0; g < nops; ++g)
    if (ops[g]->o.dim != dim || ops[g]->o.p[0] != P) {
      set_error("tdz_batch_create: all 2-D/3-D operators of a batch need the same dimension and degree");
      return TDZ_EUNSUPPORTED;
    }
  if (P < 1 || P > 8) return TDZ_EUNSUPPORTED;
  NdBatch* b = new (std::nothrow) NdBatch;
  if (!b) return TDZ_ENOMEM;
  b->prec = precision;
  b->dim = dim;
  b->P = P;
  b->nruns = nruns;
  b->st = static_cast<cudaStream_t>(stream);
  for (int g = 0; g < nops; ++g) b->ops.push_back(ops[g]->o);
  // per-geometry device tables
  struct GeoDev {
    AxisDev ax[3];
    int n[3], E[3], nq[3], Q[3];
  };
  std::vector<GeoDev> geo(nops);
  for (int g = 0; g < nops; ++g) {
    const Ops& o = ops[g]->o;
    for (int a = 0; a < dim; ++a) {
      const Basis& B = o.axis[a];
      AxisDev A{};
      A.n = (int)o.n[a];
      A.E = (int)B.nelem();
      A.nq = B.nq;
      A.Q = A.E * A.nq;
      auto up = [&](const std::vector<double>& v) -> double* {
        void* p = b->alloc(sizeof(double) * v.size());
        if (!p) return nullptr;
        cudaMemcpyAsync(p, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, b->st);
        cudaStreamSynchronize(b->st);
        return static_cast<double*>(p);
      };
      auto upf = [&](const std::vector<double>& v) -> float* {
        std::vector<float> f(v.begin(), v.end());
        void* p = b->alloc(sizeof(float) * f.size());
        if (!p) return nullptr;
        cudaMemcpyAsync(p, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice, b->st);
        cudaStreamSynchronize(b->st);
        return static_cast<float*>(p);
      };
      A.B = up(B.val);
      A.dB = up(B.der);
      A.x = up(B.xq);
      A.w = up(B.wq);
      A.S = up(o.Sa[a].a);
      A.T1 = up(o.T1a[a].a);
      A.D = up(o.Da[a].a);
      A.fB = upf(B.val);
      A.fdB = upf(B.der);
      A.fx = upf(B.xq);
      A.fw = upf(B.wq);
      A.fS = upf(o.Sa[a].a);
      A.fT1 = upf(o.T1a[a].a);
      A.fD = upf(o.Da[a].a);
      auto upl = [&](const std::vector<double>& v) -> float* {
        std::vector<double> lo(v.size());
        for (size_t k = 0; k < v.size(); ++k) lo[k] = v[k] - (double)(float)v[k];
        return upf(lo);
      };
      A.lB = upl(B.val);
      A.lx = upl(B.xq);
      A.lw = upl(B.wq);
      auto upx = [&](const std::vector<double>& v) -> fx* {
        std::vector<fx> h(v.size());
        for (size_t k = 0; k < v.size(); ++k) h[k] = fx(v[k]);
        void* p = b->alloc(sizeof(fx) * h.size());
        if (!p) return nullptr;
        cudaMemcpyAsync(p, h.data(), sizeof(fx) * h.size(), cudaMemcpyHostToDevice, b->st);
        cudaStreamSynchronize(b->st);
        return static_cast<fx*>(p);
      };
      A.xB = upx(B.val);
      A.xdB = upx(B.der);
      A.xx = upx(B.xq);
      A.xw = upx(B.wq);
      A.xS = upx(o.Sa[a].a);
      A.xT1 = upx(o.T1a[a].a);
      A.xD = upx(o.Da[a].a);
      A.Wc = nullptr;
      A.fWc = nullptr;
      A.xWc = nullptr;
      if (o.has_cap()) {
        A.Wc = up(o.Wa[a].a);
        A.fWc = upf(o.Wa[a].a);
        A.xWc = upx(o.Wa[a].a);
        if (!A.Wc || !A.fWc || !A.xWc) {
          delete b;
          return TDZ_ENOMEM;
        }
      }
      if (!A.B || !A.dB || !A.x || !A.w || !A.S || !A.T1 || !A.D || !A.fB || !A.fdB || !A.fx || !A.fw || !A.fS ||
          !A.fT1 || !A.fD || !A.lB || !A.lx || !A.lw || !A.xB || !A.xdB || !A.xx || !A.xw || !A.xS || !A.xT1 ||
          !A.xD) {
        delete b;
        return TDZ_ENOMEM;
      }
      geo[g].ax[a] = A;
      geo[g].n[a] = A.n;
      geo[g].E[a] = A.E;
      geo[g].nq[a] = A.nq;
      geo[g].Q[a] = A.Q;
    }
  }
  b->runs.resize(nruns);
  size_t maxN = 0, maxQ = 0, maxSide = 0, maxPad = 0;
  int maxn = 0;
  for (int r = 0; r < nruns; ++r) {
    const Ops& o = ops[ops_index[r]]->o;
    NdRun& R = b->runs[r];
    R.ops = ops_index[r];
    R.geo = ops_index[r];
    R.dim = dim;
    R.P = P;
    R.N = 1;
    long long NQ = 1;
    for (int a = 0; a < dim; ++a) {
      R.ax[a] = geo[R.ops].ax[a];
      R.n[a] = geo[R.ops].n[a];
      R.E[a] = geo[R.ops].E[a];
      R.nq[a] = geo[R.ops].nq[a];
      R.Q[a] = geo[R.ops].Q[a];
      R.N *= R.n[a];
      NQ *= R.Q[a];
      maxn = std::max(maxn, R.n[a]);
    }
    R.med = medium_dev(o.med);
    R.const_mass = o.med.mass_kind == TDZ_MASS_CONST;
    R.cap = o.has_cap();
    R.cm = R.const_mass ? 1.0 / o.med.mass_par[0] : 0.0;
    R.mbar = R.const_mass ? R.cm : 0.5 * (1.0 / o.med.mass_par[2] + 1.0 / o.med.mass_par[3]);
    R.c = static_cast<double2*>(b->alloc(sizeof(double2) * R.N));
    if (!R.c) {
      delete b;
      return TDZ_ENOMEM;
    }
    maxN = std::max(maxN, (size_t)R.N);
    // the largest intermediate of a Gauss-point pass: axes 0..k at the points, the others at the
    // coefficients (k <= dim - 2; the last axis is always fused), or the state itself
    size_t mq = (size_t)R.N;
    {
      size_t padded = 1;  // fast-diagonalisation planes on the grid padded to multiples of 8
      for (int a = 0; a < dim; ++a) padded *= (size_t)((R.n[a] + 7) / 8 * 8);
      mq = std::max(mq, padded);
      maxPad = std::max(maxPad, padded);
    }
    for (int k = 0; k + 1 < dim; ++k) {
      size_t part = 1;
      for (int a = 0; a < dim; ++a) part *= (size_t)(a <= k ? R.Q[a] : R.n[a]);
      mq = std::max(mq, part);
    }
    maxQ = std::max(maxQ, mq);
    {
      long long inner = 1;
      for (int a = 0; a + 1 < dim; ++a) inner *= R.Q[a];
      int ec = 1;
      const long long nch = fused_nchunks(R.E[dim - 1], inner, P, &ec);
      maxSide = std::max(maxSide, (size_t)((nch - 1) * P * inner));
    }
    (void)NQ;
  }
  b->maxN = maxN;
  b->maxQ = maxQ;
  b->maxPad = maxPad;
  b->maxSide = maxSide;
  b->maxn = maxn;
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
      b->nsm = nsm;
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) b->dev_name = prop.name;
  }
  const size_t before_work = b->dev_bytes;
  const bool work_ok = alloc_work(b);
  b->work_bytes = b->dev_bytes - before_work;
  if (!work_ok) {
    delete b;
    set_error("tdz_batch_create: device allocation for 2-D/3-D work buffers failed");
    return TDZ_ENOMEM;
  }
  // per geometry: fast-diagonalisation factors and (2-D) the assembled stencil
  b->geo.resize(nops);
  if (cublasCreate(&b->blas) != CUBLAS_STATUS_SUCCESS || cublasSetStream(b->blas, b->st) != CUBLAS_STATUS_SUCCESS) {
    delete b;
    set_error("tdz_batch_create: cuBLAS initialisation failed");
    return TDZ_ECUDA;
  }
  // cuBLAS serves only the binary64 path's fast-diagonalisation DGEMMs; the mixed path's transforms are
  // the library's own tensor-core kernel (tdz_tc.cu)
  size_t stencil_bytes = 0;
  if (dim == 2)
    for (int g = 0; g < nops; ++g)
      stencil_bytes += (size_t)geo[g].n[0] * geo[g].n[1] *
                       (precision == TDZ_MIXED ? half_count(P) * sizeof(fx) + (2 * P + 1) * (2 * P + 1) * sizeof(float)
                                               : half_count(P) * sizeof(double));
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const bool want_stencil = dim == 2 && stencil_bytes < free_b / 2;
  for (int g = 0; g < nops; ++g) {
    const int rc = fd_setup(b, g, ops[g]->o);
    if (rc == TDZ_ENOMEM) {
      delete b;
      return rc;
    }
    if (want_stencil) {
      const int rs = stencil_setup(b, g, geo[g].ax[0], geo[g].ax[1], medium_dev(ops[g]->o.med),
                                   ops[g]->o.med.mass_kind != TDZ_MASS_CONST);
      if (rs != TDZ_OK) {
        delete b;
        return rs;
      }
    }
  }
  // 3-D mixed batches: tabulate w V at the Gauss points for the double-float passes when the device has
  // room for it (8 bytes per point, at most half of the free memory); otherwise V is evaluated per point
  if (dim == 3 && precision == TDZ_MIXED) {
    size_t need = 0;
    for (int g = 0; g < nops; ++g)
      if (ops[g]->o.med.pot_kind != TDZ_POT_ZERO)
        need += (size_t)geo[g].Q[0] * geo[g].Q[1] * geo[g].Q[2] * sizeof(fx);
    cudaMemGetInfo(&free_b, &total_b);
    if (need > 0 && need < free_b / 2) {
      for (int g = 0; g < nops; ++g) {
        if (ops[g]->o.med.pot_kind == TDZ_POT_ZERO) continue;
        const size_t nq3 = (size_t)geo[g].Q[0] * geo[g].Q[1] * geo[g].Q[2];
        b->geo[g].Vqx = static_cast<fx*>(b->alloc(sizeof(fx) * nq3));
        if (!b->geo[g].Vqx) {
          delete b;
          set_error("tdz_batch_create: device allocation for the 3-D potential table failed");
          return TDZ_ENOMEM;
        }
        k_vtab3<<<grid_for((long long)nq3), TPB, 0, b->st>>>(geo[g].ax[0], geo[g].ax[1], geo[g].ax[2],
                                                             medium_t<double>(medium_dev(ops[g]->o.med)),
                                                             b->geo[g].Vqx);
      }
    }
  }
  // soft-core geometries of constant mass (both precisions): tabulate the observables' point factor
  // w m^-1 Z (r^2 + eps)^(-3/2) when the device has room (8 bytes per point, at most half of the free
  // memory); otherwise the gradient is evaluated per point in double-float
  for (int g = 0; g < nops; ++g) {
    const Medium& md = ops[g]->o.med;
    if (md.pot_kind != TDZ_POT_SOFTCORE || md.mass_kind != TDZ_MASS_CONST) continue;
    const size_t npts = (size_t)geo[g].Q[0] * geo[g].Q[1] * (dim > 2 ? geo[g].Q[2] : 1);
    cudaMemGetInfo(&free_b, &total_b);
    if (npts * sizeof(fx) >= free_b / 2) continue;
    b->geo[g].Gq = static_cast<fx*>(b->alloc(sizeof(fx) * npts));
    if (!b->geo[g].Gq) continue;
    k_gtab<<<grid_for((long long)npts), TPB, 0, b->st>>>(geo[g].ax[0], geo[g].ax[1], geo[g].ax[dim > 2 ? 2 : 1], dim,
                                                         md.pot_par[0] / md.mass_par[0], md.pot_par[1], b->geo[g].Gq);
  }
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) {
    delete b;
    return nd_cuda_fail(e, "tdz_batch_create (2-D/3-D)");
  }
  if (dim == 2 && precision == TDZ_MIXED && want_stencil && autotune(b) != TDZ_OK) {
    delete b;
    set_error("tdz_batch_create: timing the 2-D apply variants failed");
    return TDZ_ECUDA;
  }
  if (precision == TDZ_MIXED && autotune_fd(b) != TDZ_OK) {
    delete b;
    set_error("tdz_batch_create: timing the tensor-core preconditioner transforms failed");
    return TDZ_ECUDA;
  }
  const int rw = make_workers(b);
  if (rw != TDZ_OK) {
    delete b;
    set_error("tdz_batch_create: creating the 2-D/3-D workers failed");
    return rw;
  }
  *out = b;
  return TDZ_OK;
}

void nd_batch_destroy(NdBatch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->st);
  delete b;
}

long long nd_run_size(const NdBatch* b, int run) { return b->runs[run].N; }

int nd_set_state(NdBatch* b, int run, const double* c, bool device) {
  NdRun& R = b->runs[run];
  cudaError_t e = cudaMemcpyAsync(R.c, c, sizeof(double2) * R.N, device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return nd_cuda_fail(e, "tdz_set_state");
  R.status = TDZ_OK;
  return TDZ_OK;
}

int nd_get_state(const NdBatch* b, int run, double* c, bool device) {
  const NdRun& R = b->runs[run];
  cudaError_t e = cudaMemcpyAsync(c, R.c, sizeof(double2) * R.N, device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return nd_cuda_fail(e, "tdz_get_state");
  return TDZ_OK;
}

// One apply of the inner-solve operator y = A_n x (FP32 in mixed batches, binary64 otherwise) for run r,
// on the batch's work buffers, timed with CUDA events: best of `reps` after one warm-up apply.
template <int P>
int time_operator_p(NdBatch* b, NdRun* r, int reps, double* ms_out) {
  const NdGeo& G = b->geo[r->geo];
  const bool stencil = G.has_stencil() && b->opt_operator != TDZ_OPERATOR_QUADRATURE;
  const double tau = 0.025, ebar[3] = {0.01, 0.01, 0.01};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return TDZ_ECUDA;
  }
  float best = 0.f;
  cudaError_t e = cudaSuccess;
  auto timed = [&](auto&& apply_once) {
    apply_once();
    for (int k = 0; k < reps && e == cudaSuccess; ++k) {
      cudaEventRecord(e0, b->st);
      apply_once();
      cudaEventRecord(e1, b->st);
      float ms = 0.f;
      e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      best = k == 0 ? ms : std::min(best, ms);
    }
  };
  if (b->prec == TDZ_MIXED) {
    Apply<float, P> op{b, r, static_cast<C<float>*>(b->w_t1), static_cast<C<float>*>(b->w_t2),
                       static_cast<C<float>*>(b->w_t3), static_cast<C<float>*>(b->w_t4),
                       static_cast<C<float>*>(b->w_qa), static_cast<C<float>*>(b->w_qb)};
    if (stencil) op.Wm = r->cap ? nullptr : G.W32;
    op.Vtab = nullptr;  // the FP32 apply evaluates the potential at the points
    const C<float>* x = static_cast<const C<float>*>(b->w_p);
    C<float>* y = static_cast<C<float>*>(b->w_q);
    timed([&]() { op.apply(x, y, tau, ebar); });
  } else {
    Apply<double, P> op{b, r, reinterpret_cast<C<double>*>(b->d_t1), reinterpret_cast<C<double>*>(b->d_t2),
                        reinterpret_cast<C<double>*>(b->d_t3), reinterpret_cast<C<double>*>(b->d_t4),
                        reinterpret_cast<C<double>*>(b->d_qa), reinterpret_cast<C<double>*>(b->d_qb)};
    if (stencil) op.Wm = G.W64;
    const C<double>* x = reinterpret_cast<const C<double>*>(b->d_p);
    C<double>* y = reinterpret_cast<C<double>*>(b->d_q);
    timed([&]() { op.apply(x, y, tau, ebar); });
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->rb_geo = -1;
  if (e != cudaSuccess) return nd_cuda_fail(e, "tdz_batch_time_operator");
  int werr = 0;
  if (cudaMemcpy(&werr, b->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || werr != 0) return TDZ_ECUDA;
  *ms_out = best;
  return TDZ_OK;
}

int nd_ground_state(NdBatch* b, int run, double sigma, double tol, int max_outer, double* energy, int* outer,
                    double* resid) {
  if (!b || run < 0 || run >= b->nruns || !(tol > 0.0) || max_outer < 1) return TDZ_EINVAL;
  NdRun* r = &b->runs[run];
  if (r->cap || !use_fd(b, r)) {
    set_error("tdz_batch_ground_state: needs the fast-diagonalisation preconditioner and no absorbing layer");
    return TDZ_EUNSUPPORTED;
  }
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return nd_cuda_fail(e, "tdz_batch_ground_state");
  if (b->prec == TDZ_MIXED) {
    switch (b->P) {
      case 1: return ground_state_run<float, 1>(b, r, sigma, tol, max_outer, energy, outer, resid);
      case 2: return ground_state_run<float, 2>(b, r, sigma, tol, max_outer, energy, outer, resid);
      case 3: return ground_state_run<float, 3>(b, r, sigma, tol, max_outer, energy, outer, resid);
      case 4: return ground_state_run<float, 4>(b, r, sigma, tol, max_outer, energy, outer, resid);
      case 5: return ground_state_run<float, 5>(b, r, sigma, tol, max_outer, energy, outer, resid);
      case 6: return ground_state_run<float, 6>(b, r, sigma, tol, max_outer, energy, outer, resid);
      case 7: return ground_state_run<float, 7>(b, r, sigma, tol, max_outer, energy, outer, resid);
      default: return ground_state_run<float, 8>(b, r, sigma, tol, max_outer, energy, outer, resid);
    }
  }
  switch (b->P) {
    case 1: return ground_state_run<double, 1>(b, r, sigma, tol, max_outer, energy, outer, resid);
    case 2: return ground_state_run<double, 2>(b, r, sigma, tol, max_outer, energy, outer, resid);
    case 3: return ground_state_run<double, 3>(b, r, sigma, tol, max_outer, energy, outer, resid);
    case 4: return ground_state_run<double, 4>(b, r, sigma, tol, max_outer, energy, outer, resid);
    case 5: return ground_state_run<double, 5>(b, r, sigma, tol, max_outer, energy, outer, resid);
    case 6: return ground_state_run<double, 6>(b, r, sigma, tol, max_outer, energy, outer, resid);
    case 7: return ground_state_run<double, 7>(b, r, sigma, tol, max_outer, energy, outer, resid);
    default: return ground_state_run<double, 8>(b, r, sigma, tol, max_outer, energy, outer, resid);
  }
}

int nd_time_operator(NdBatch* b, int geometry, int reps, double* ms) {
  if (geometry < 0 || geometry >= (int)b->geo.size() || reps < 1 || !ms) return TDZ_EINVAL;
  NdRun* r = nullptr;
  for (auto& run : b->runs)
    if (run.geo == geometry) {
      r = &run;
      break;
    }
  if (!r) return TDZ_EINVAL;
  switch (b->P) {
    case 1: return time_operator_p<1>(b, r, reps, ms);
    case 2: return time_operator_p<2>(b, r, reps, ms);
    case 3: return time_operator_p<3>(b, r, reps, ms);
    case 4: return time_operator_p<4>(b, r, reps, ms);
    case 5: return time_operator_p<5>(b, r, reps, ms);
    case 6: return time_operator_p<6>(b, r, reps, ms);
    case 7: return time_operator_p<7>(b, r, reps, ms);
    default: return time_operator_p<8>(b, r, reps, ms);
  }
}

static int propagate_one(NdBatch* w, NdBatch* b, int r, const double* field_host, double dt, long long step0,
                         long long nsteps) {
  const int D = b->dim, cols = 2 + 3 * D;
  NdRun& R = b->runs[r];
  const double* f = field_host + (size_t)r * (nsteps + 1) * D;
  double* o = &b->obs[(size_t)r * nsteps * cols];
  const Ops& ops = b->ops[R.ops];
  switch (b->P) {
    case 1: return propagate_run<1>(w, &R, ops, f, dt, step0, nsteps, o);
    case 2: return propagate_run<2>(w, &R, ops, f, dt, step0, nsteps, o);
    case 3: return propagate_run<3>(w, &R, ops, f, dt, step0, nsteps, o);
    case 4: return propagate_run<4>(w, &R, ops, f, dt, step0, nsteps, o);
    case 5: return propagate_run<5>(w, &R, ops, f, dt, step0, nsteps, o);
    case 6: return propagate_run<6>(w, &R, ops, f, dt, step0, nsteps, o);
    case 7: return propagate_run<7>(w, &R, ops, f, dt, step0, nsteps, o);
    default: return propagate_run<8>(w, &R, ops, f, dt, step0, nsteps, o);
  }
}

// Runs are independent: with workers, host threads take runs longest first from a shared counter,
// each on its own worker (stream, handle, buffers); the call returns when all runs are done.
int nd_propagate(NdBatch* b, const double* field_host, double dt, long long step0, long long nsteps) {
  const int D = b->dim;
  const int cols = 2 + 3 * D;
  b->obs.assign((size_t)b->nruns * nsteps * cols, 0.0);
  b->last_nsteps = 0;  // set again when the call succeeds (tdz_observe then reads the new buffer)
  const int nw = (int)std::min<size_t>(b->workers.size() + 1, (size_t)b->nruns);
  if (nw <= 1) {
    for (int r = 0; r < b->nruns; ++r) {
      const int rc = propagate_one(b, b, r, field_host, dt, step0, nsteps);
      if (rc != TDZ_OK) return rc;
    }
    b->last_nsteps = nsteps;
    return TDZ_OK;
  }
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return nd_cuda_fail(e, "tdz_propagate (2-D/3-D)");
  for (NdBatch* w : b->workers) {  // solver settings may have changed since creation
    w->tol = b->tol;
    w->max_it = b->max_it;
    w->inner_tol = b->inner_tol;
    w->opt_precond = b->opt_precond;
    w->opt_operator = b->opt_operator;
    w->opt_groups = b->opt_groups;
    w->opt_wait_test = b->opt_wait_test;
  }
  std::vector<int> order(b->nruns);
  for (int r = 0; r < b->nruns; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->runs[x].N > b->runs[y].N; });
  int dev = 0;
  cudaGetDevice(&dev);
  std::atomic<int> next(0);
  std::vector<int> rcs(nw, TDZ_OK);
  std::vector<std::thread> th;
  for (int t = 0; t < nw; ++t) {
    th.emplace_back([&, t]() {
      cudaSetDevice(dev);
      NdBatch* w = t == 0 ? b : b->workers[t - 1];
      for (int k = next++; k < b->nruns; k = next++) {
        const int rc = propagate_one(w, b, order[k], field_host, dt, step0, nsteps);
        if (rc != TDZ_OK) {
          rcs[t] = rc;
          break;
        }
      }
      if (cudaStreamSynchronize(w->st) != cudaSuccess && rcs[t] == TDZ_OK) rcs[t] = TDZ_ECUDA;
    });
  }
  for (auto& x : th) x.join();
  for (int rc : rcs)
    if (rc != TDZ_OK) return rc;
  b->last_nsteps = nsteps;
  return TDZ_OK;
}

int nd_observe(const NdBatch* b, int run, double* out, int* status, bool device) {
  const int cols = 2 + 3 * b->dim;
  const size_t cnt = (size_t)b->last_nsteps * cols;
  if (out && cnt) {
    cudaError_t e = cudaMemcpy(out, &b->obs[(size_t)run * cnt], sizeof(double) * cnt,
                               device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost);
    if (e != cudaSuccess) return nd_cuda_fail(e, "tdz_observe");
  }
  if (status) *status = b->runs[run].status;
  return TDZ_OK;
}

int nd_stats(const NdBatch* b, double* max_rel, double* solves, double* iters) {
  double mx = 0, ns = 0, it = 0;
  for (const auto& r : b->runs) {
    mx = std::max(mx, r.max_rel);
    ns += (double)r.nsolve;
    it += (double)r.iters;
  }
  if (max_rel) *max_rel = mx;
  if (solves) *solves = ns;
  if (iters) *iters = it;
  return TDZ_OK;
}

int nd_set_option(NdBatch* b, int option, int value) {
  if (option == TDZ_OPT_PRECOND) {
    if (value < TDZ_PRECOND_AUTO || value > TDZ_PRECOND_FD) return TDZ_EINVAL;
    if (value == TDZ_PRECOND_FD)
      for (const auto& g : b->geo)
        if (!g.fd) {
          set_error("tdz_batch_set_option: fast diagonalisation is not set up for this batch");
          return TDZ_EUNSUPPORTED;
        }
    b->opt_precond = value;
    return TDZ_OK;
  }
  if (option == TDZ_OPT_OPERATOR) {
    if (value < TDZ_OPERATOR_AUTO || value > TDZ_OPERATOR_STENCIL) return TDZ_EINVAL;
    if (value == TDZ_OPERATOR_STENCIL)
      for (const auto& g : b->geo)
        if (!g.has_stencil()) {
          set_error("tdz_batch_set_option: the stencil operator exists for 2-D batches with enough device memory");
          return TDZ_EUNSUPPORTED;
        }
    b->opt_operator = value;
    return TDZ_OK;
  }
  if (option == TDZ_OPT_APPLY_GROUPS) {
    if (value != 0 && value != 8 && value != 16) return TDZ_EINVAL;
    b->opt_groups = value;
    return TDZ_OK;
  }
  if (option == TDZ_OPT_WAIT_TEST) {
    if (value != 0 && value != 1) return TDZ_EINVAL;
    b->opt_wait_test = value;
    return TDZ_OK;
  }
  return TDZ_EINVAL;
}

int nd_precond_tuning(const NdBatch* b, int geometry, int* variant, double* ms) {
  if (geometry < 0 || geometry >= (int)b->geo.size()) return TDZ_EINVAL;
  const NdGeo& G = b->geo[geometry];
  const bool tuned = G.fd && G.Vt[0] && G.tc_variant >= 0;
  if (variant) *variant = tuned ? G.tc_variant : -1;
  if (ms)
    for (int c = 0; c < 6; ++c) ms[c] = tuned ? G.tc_ms[c] : 0.0;
  return TDZ_OK;
}

int nd_tuning(const NdBatch* b, int geometry, int* groups, double* ms) {
  if (geometry < 0 || geometry >= (int)b->geo.size()) return TDZ_EINVAL;
  const NdGeo& G = b->geo[geometry];
  if (!G.W32) {
    if (groups) *groups = 0;
    if (ms) ms[0] = ms[1] = 0.0;
    return TDZ_OK;
  }
  if (groups) *groups = G.apply_groups;
  if (ms) {
    ms[0] = G.tune_ms[0];
    ms[1] = G.tune_ms[1];
  }
  return TDZ_OK;
}

void nd_set_refinement(NdBatch* b, double tol, int max_it) {
  b->tol = tol;
  b->max_it = std::max(max_it, 50);
}

}  // namespace tdz

namespace tdz {
int nd_dim(const NdBatch* b) { return b->dim; }
size_t nd_device_bytes(const NdBatch* b) {
  size_t t = b->dev_bytes;
  for (const NdBatch* w : b->workers) t += w->dev_bytes;
  return t;
}
}  // namespace tdz
