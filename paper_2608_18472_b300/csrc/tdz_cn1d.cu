// Batched 1-D Crank-Nicolson propagation on sm_103a.
//
// Method (arXiv 2608.18472, Sec. "Time propagation", Eq. cn_system): per step
//     (S + i tau H_n) c^{n+1} = (S - i tau H_n) c^n,  tau = dt/2,  H_n = H0 + Ebar_n D,
// solved here in correction form: c^{n+1} = y0 + delta with
//     A_n delta = r,  r = B_n c^n - A_n y0 = -S w - i tau H_n (2 c^n + w),  w = y0 - c^n,
// where A_n = S + i tau H_n is complex symmetric with positive definite Hermitian part S,
// so an unpivoted LDL^T factorisation is stable. y0 = c^n (binary64 path) or a quadratic
// extrapolation from the last two steps (mixed path). Observables of Sec. "Dipoles" are
// reduced after every step.
//
// GPU organisation (the whole time loop inside one persistent launch):
//   * the n rows of a run are split into K chunks of m rows, one per lane, K chosen on the host so that
//     every run of the batch has about the same m; the runs are packed lane by lane into blocks (a run's
//     K lanes are consecutive threads of one block, and may span warps); the last P rows of every chunk
//     but the last are a separator ("Sep_k"), the rest its interior;
//   * sweep 1 (top-down): each lane eliminates its interior with a register-window band
//     LDL^T, carrying the coupling to the separator above (the "spike") and the right-hand
//     side; it stores L and D^-1 and leaves the Schur complement of its lower separator;
//   * sweep 2 (bottom-up): each lane eliminates its interior from the bottom to obtain the
//     Schur complement of the separator above it (no storage);
//   * the separators form a block-tridiagonal system (K-1 blocks of P x P), kept in the shared memory of
//     the run's own lanes and factored and solved by the warp that holds the run's first lane (block
//     LDL^T with explicit pivot inverses);
//   * forward/back substitution of every interior with the separator values;
//   * state update and observables.
// All arrays of a run are interleaved [row][lane of the run] so that every warp access is coalesced.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tdz_arith.cuh"
#include "tdz_internal.h"

namespace tdz {

constexpr int LANES = 32;
constexpr int MAXP = 8;

struct GeomDev {
  int n, m, K;
  int ks;  // interleave stride of the per-row arrays: the run's lanes (K)
  // Band arrays, [m][P+1][32] each.
  //   binary64 path: S, H (= H0 = T + V), D, G, Km (<m^-1>) as double.
  //   mixed path:    S  = float4 {S.hi, H0.hi, D.hi, S.lo}   (one 16-byte load per entry in the sweeps)
  //                  H  = float2 {H0.lo, D.lo}
  //                  G  = float4 {G.hi, G.lo, K.hi, K.lo};  D and Km unused.
  const void* S;
  const void* H;
  const void* D;
  const void* G;
  const void* Km;
  // absorbing-layer mask W (the real band of the CAP matrix), [m][P+1][32] like the others; null without a
  // layer. binary64 path: double; mixed path: float2 {W.hi, W.lo}.
  const void* Wc;
  // lower band of the velocity matrix's antisymmetric part M (Vel = -(i/2) M), same layout and types as Wc;
  // null unless the batch records the current
  const void* Mv;
};

struct RunDev {
  int geom;
  int status;
  int hist;        // steps of valid difference history (mixed)
  int pad;
  void* state;     // binary64: double2 [m][32]; mixed: float4 {hr, hi, lr, li} [m][32]
  float2* d1;      // mixed: c^n - c^{n-1}
  float2* d2;      // mixed: c^{n-1} - c^{n-2}
  float4* W;       // mixed: correction w (double-float complex)
  void* rhs;       // cx<T> [m][32]
  void* Lc;        // cx<T> [m][P][32]
  void* Dv;        // cx<T> [m][32]
  void* gd;        // cx<T> [m][32]
  void* dl;        // cx<T> [m][32]
  double max_rel;  // largest final relative residual (mixed)
  long long nsolve;
};

struct StepArgs {
  const GeomDev* geoms;
  RunDev* runs;
  const int* lanes;  // [ngroups][threads per block]: run << 8 | lane of the run, or -1 (no run)
  int ngroups;
  int* counter;
  const double* field;  // [run][nsteps+1]
  double* obs;          // [run][nsteps][5]
  double* cur;          // [run][nsteps] total dipole velocity J = c^H Vel c, or null
  long long nsteps;
  long long step0;
  double dt;
  double tol;
  int max_it;
};

// ============================================================================ band access
template <int P>
TDZ_DEV int bidx(int i, int d, int k, int ks) { return (i * (P + 1) + d) * ks + k; }
TDZ_DEV int ridx(int i, int k, int ks) { return i * ks + k; }
// L1 prefetch of the line holding p: rows ahead of a lane's sequential row loop are requested
// early, so the loop does not pay a full memory round trip per row (no registers needed).
TDZ_DEV void pf(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// A(i, i-d) entry for the factorisation, in the solve precision T: S + tau W + i tau (H0 + Ebar D), the
// absorbing layer's tau W only when CAP.
template <int P, class T, bool MIXED, bool CAP>
TDZ_DEV cx<T> a_entry(const GeomDev& g, int idx, T tau, T ebar) {
  if constexpr (MIXED) {
    const float4 v = __ldg(static_cast<const float4*>(g.S) + idx);
    float re = v.x;
    if constexpr (CAP) re = fmaf(tau, __ldg(static_cast<const float2*>(g.Wc) + idx).x, re);
    return cx<T>{re, tau * fmaf(ebar, v.z, v.y)};
  } else {
    double s = __ldg(static_cast<const double*>(g.S) + idx);
    const double h = __ldg(static_cast<const double*>(g.H) + idx);
    const double d = __ldg(static_cast<const double*>(g.D) + idx);
    if constexpr (CAP) s = fma(tau, __ldg(static_cast<const double*>(g.Wc) + idx), s);
    return cx<T>{s, tau * fma(ebar, d, h)};
  }
}

// ============================================================================ per-lane context
struct Lane {
  int k, K, m, mI, ks;  // chunk index, chunks, rows per chunk, interior rows, interleave stride
  bool active, up, dn;
};

// Shared memory of a block (elements of the solve precision's complex type, then doubles):
//   * per lane 2 P^2 + P: a run of K lanes keeps its K - 1 separators' Dg and E blocks and rb vectors in
//     the area of its own lanes;
//   * per warp one P x P scratch tile for the reduced factorisation the warp runs;
//   * per lane 2 x 5 doubles for the run sums.
__host__ __device__ constexpr int red_lane_elems(int P) { return 2 * P * P + P; }

template <class T>
struct Red {  // reduced system of one run in shared memory
  cx<T>* Dg;  // [31][P*P]  diagonal blocks -> pivot inverses
  cx<T>* E;   // [31][P*P]  sub-diagonal blocks Ŝ(s, s-1) -> F_s
  cx<T>* rb;  // [31][P]    rhs -> separator solution
  cx<T>* Wt;  // [P*P]      scratch tile
};

// ============================================================================ sweep 1 (top-down)
// Eliminates the interior rows 0..mI-1 of the lane's chunk. Stores L (column-wise: Lc[i][d-1]
// = L(i+d, i)) and D^-1, and returns in registers the Schur complement of the rows mI..mI+P-1
// (the lane's separator), their coupling to the separator above and their reduced rhs.
template <int P, class T, bool MIXED, bool CAP>
TDZ_DEV void sweep1(const GeomDev& g, const RunDev& run, const Lane& L, T tau, T ebar, Red<T>& red) {
  const int ks = L.ks;
  cx<T> w[P + 1][P + 1];
  cx<T> cw[P + 1][P];
  cx<T> rw[P + 1];
  const cx<T>* rhs = static_cast<const cx<T>*>(run.rhs);
  cx<T>* Lc = static_cast<cx<T>*>(run.Lc);
  cx<T>* Dv = static_cast<cx<T>*>(run.Dv);
  const int k = L.k;
#pragma unroll
  for (int a = 0; a < P; ++a) {
#pragma unroll
    for (int b = 0; b <= a; ++b) w[a][b] = a_entry<P, T, MIXED, CAP>(g, bidx<P>(a, a - b, k, ks), tau, ebar);
#pragma unroll
    for (int j = 0; j < P; ++j)
      cw[a][j] = (L.up && a <= j) ? a_entry<P, T, MIXED, CAP>(g, bidx<P>(a, a + P - j, k, ks), tau, ebar) : czero<T>();
    rw[a] = rhs[ridx(a, k, ks)];
  }
  for (int i = 0; i < L.mI; ++i) {
    const int r = i + P;  // row entering the window
    if (r + 2 < L.m) {
#pragma unroll
      for (int b = 0; b <= P; ++b) pf(static_cast<const char*>(g.S) + (size_t)bidx<P>(r + 2, b, k, ks) * (MIXED ? 16 : 8));
      pf(rhs + ridx(r + 2, k, ks));
    }
    if (r < L.m) {
#pragma unroll
      for (int b = 0; b <= P; ++b) w[P][b] = a_entry<P, T, MIXED, CAP>(g, bidx<P>(r, P - b, k, ks), tau, ebar);
      rw[P] = rhs[ridx(r, k, ks)];
    } else {
#pragma unroll
      for (int b = 0; b <= P; ++b) w[P][b] = czero<T>();
      rw[P] = czero<T>();
    }
#pragma unroll
    for (int j = 0; j < P; ++j) cw[P][j] = czero<T>();
    const cx<T> dinv = crecip(w[0][0]);
    cx<T> l[P + 1];
#pragma unroll
    for (int a = 1; a <= P; ++a) {
      l[a] = cmul(w[a][0], dinv);
      Lc[(i * P + a - 1) * ks + k] = l[a];
    }
    Dv[ridx(i, k, ks)] = dinv;
#pragma unroll
    for (int a = 1; a <= P; ++a) {
#pragma unroll
      for (int b = 1; b <= a; ++b) w[a][b] = cmsub(w[a][b], l[a], w[b][0]);
#pragma unroll
      for (int j = 0; j < P; ++j) cw[a][j] = cmsub(cw[a][j], l[a], cw[0][j]);
      rw[a] = cmsub(rw[a], l[a], rw[0]);
    }
#pragma unroll
    for (int a = 0; a < P; ++a) {
#pragma unroll
      for (int b = 0; b <= a; ++b) w[a][b] = w[a + 1][b + 1];
#pragma unroll
      for (int j = 0; j < P; ++j) cw[a][j] = cw[a + 1][j];
      rw[a] = rw[a + 1];
    }
  }
  if (L.dn) {
    cx<T>* Dg = red.Dg + k * P * P;
    cx<T>* E = red.E + k * P * P;
#pragma unroll
    for (int a = 0; a < P; ++a) {
#pragma unroll
      for (int b = 0; b <= a; ++b) {
        Dg[a * P + b] = w[a][b];
        Dg[b * P + a] = w[a][b];
      }
#pragma unroll
      for (int j = 0; j < P; ++j) E[a * P + j] = cw[a][j];
      red.rb[k * P + a] = rw[a];
    }
  }
}

// ============================================================================ sweep 2 (bottom-up)
// Eliminates the interior from its last row upwards with the separator above (rows -P..-1)
// entering with zero self block and zero rhs: what remains is -C^T A_II^-1 C and -C^T A_II^-1 b
// for that separator; added into the shared reduced system.
template <int P, class T, bool MIXED, bool CAP>
TDZ_DEV void sweep2(const GeomDev& g, const RunDev& run, const Lane& L, T tau, T ebar, Red<T>& red) {
  const int ks = L.ks;
  cx<T> w[P + 1][P + 1];  // w[a][b] = A(r-a, r-b), b <= a, r = current pivot row
  cx<T> rw[P + 1];
  const cx<T>* rhs = static_cast<const cx<T>*>(run.rhs);
  const int k = L.k;
  const int r0 = L.mI - 1;
#pragma unroll
  for (int a = 0; a < P; ++a) {
#pragma unroll
    for (int b = 0; b <= a; ++b) w[a][b] = a_entry<P, T, MIXED, CAP>(g, bidx<P>(r0 - b, a - b, k, ks), tau, ebar);
    rw[a] = rhs[ridx(r0 - a, k, ks)];
  }
  for (int t = 0; t < L.mI; ++t) {
    const int r = r0 - t;
    const int q = r - P;  // row entering the window
    if (q - 2 >= 0) {
#pragma unroll
      for (int b = 0; b <= P; ++b) pf(static_cast<const char*>(g.S) + (size_t)bidx<P>(q - 2, b, k, ks) * (MIXED ? 16 : 8));
      pf(rhs + ridx(q - 2, k, ks));
    }
#pragma unroll
    for (int b = 0; b <= P; ++b) {
      const int rb = r - b;  // A(q, rb) stored at row rb (rb >= q), diagonal P - b
      w[P][b] = (rb >= 0) ? a_entry<P, T, MIXED, CAP>(g, bidx<P>(rb, P - b, k, ks), tau, ebar) : czero<T>();
    }
    rw[P] = (q >= 0) ? rhs[ridx(q, k, ks)] : czero<T>();
    const cx<T> dinv = crecip(w[0][0]);
    cx<T> l[P + 1];
#pragma unroll
    for (int a = 1; a <= P; ++a) l[a] = cmul(w[a][0], dinv);
#pragma unroll
    for (int a = 1; a <= P; ++a) {
#pragma unroll
      for (int b = 1; b <= a; ++b) w[a][b] = cmsub(w[a][b], l[a], w[b][0]);
      rw[a] = cmsub(rw[a], l[a], rw[0]);
    }
#pragma unroll
    for (int a = 0; a < P; ++a) {
#pragma unroll
      for (int b = 0; b <= a; ++b) w[a][b] = w[a + 1][b + 1];
      rw[a] = rw[a + 1];
    }
  }
  // window rows -1..-P  <->  separator (k-1) local index j = P-1-a
  cx<T>* Dg = red.Dg + (k - 1) * P * P;
#pragma unroll
  for (int a = 0; a < P; ++a) {
    const int ja = P - 1 - a;
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      const int jb = P - 1 - b;
      Dg[ja * P + jb] = Dg[ja * P + jb] + w[a][b];
      if (ja != jb) Dg[jb * P + ja] = Dg[jb * P + ja] + w[a][b];
    }
    red.rb[(k - 1) * P + ja] = red.rb[(k - 1) * P + ja] + rw[a];
  }
}

// ============================================================================ reduced system
// Lower-triangle pair number t (row-wise, 0 <= t < P(P+1)/2) -> (i, j), i >= j.
TDZ_DEV void tri_pair(int t, int& i, int& j) {
  i = 0;
  while (t > i) {
    t -= i + 1;
    ++i;
  }
  j = t;
}

// In-place inverse of a complex symmetric P x P block (no pivoting) by the symmetric sweep operator: sweeping
// pivot k replaces a_kk by -1/a_kk, a_ik and a_ki by a_ik / a_kk and every other a_ij by a_ij - a_ik a_kj /
// a_kk; the matrix stays symmetric throughout and all P sweeps leave -A^-1. Only the P(P+1)/2 entries of
// the lower triangle are computed (one per lane) and written to both halves.
template <int P, class T>
TDZ_DEV void red_invert(cx<T>* M, int lane) {
  constexpr int NT = P * (P + 1) / 2;
  constexpr int R = (NT + LANES - 1) / LANES;
  int ti[R], tj[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    ti[u] = tj[u] = 0;
    if (lane + u * LANES < NT) tri_pair(lane + u * LANES, ti[u], tj[u]);
  }
  for (int k = 0; k < P; ++k) {
    cx<T> nv[R];
    const cx<T> piv = crecip(M[k * P + k]);
#pragma unroll
    for (int u = 0; u < R; ++u) {
      if (lane + u * LANES < NT) {
        const int i = ti[u], j = tj[u];
        if (i == k && j == k) nv[u] = czero<T>() - piv;
        else if (i == k) nv[u] = cmul(M[j * P + k], piv);
        else if (j == k) nv[u] = cmul(M[i * P + k], piv);
        else nv[u] = cmsub(M[i * P + j], cmul(M[i * P + k], piv), M[j * P + k]);
      }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < R; ++u)
      if (lane + u * LANES < NT) M[ti[u] * P + tj[u]] = M[tj[u] * P + ti[u]] = nv[u];
    __syncwarp();
  }
#pragma unroll
  for (int u = 0; u < R; ++u)
    if (lane + u * LANES < NT) {
      const cx<T> v = czero<T>() - M[ti[u] * P + tj[u]];
      M[ti[u] * P + tj[u]] = M[tj[u] * P + ti[u]] = v;
    }
  __syncwarp();
}

template <int P, class T>
TDZ_DEV void red_factor(Red<T>& red, int nsep, int lane) {
  constexpr int NT = P * (P + 1) / 2;
  constexpr int R = (NT + LANES - 1) / LANES;
  int ti[R], tj[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    ti[u] = tj[u] = 0;
    if (lane + u * LANES < NT) tri_pair(lane + u * LANES, ti[u], tj[u]);
  }
  for (int s = 0; s < nsep; ++s) {
    cx<T>* D = red.Dg + s * P * P;
    if (s > 0) {
      const cx<T>* Pinv = red.Dg + (s - 1) * P * P;
      cx<T>* E = red.E + s * P * P;
      // F = E * Pinv
      for (int t = lane; t < P * P; t += LANES) {
        int r = t / P, c = t % P;
        cx<T> acc = czero<T>();
#pragma unroll
        for (int q = 0; q < P; ++q) acc = cmadd(acc, E[r * P + q], Pinv[q * P + c]);
        red.Wt[t] = acc;
      }
      __syncwarp();
      // D -= F * E^T (symmetric: the lower triangle, mirrored); E <- F
      cx<T> nv[R];
#pragma unroll
      for (int u = 0; u < R; ++u) {
        if (lane + u * LANES < NT) {
          const int r = ti[u], c = tj[u];
          cx<T> acc = D[r * P + c];
#pragma unroll
          for (int q = 0; q < P; ++q) acc = cmsub(acc, red.Wt[r * P + q], E[c * P + q]);
          nv[u] = acc;
        }
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < R; ++u)
        if (lane + u * LANES < NT) D[ti[u] * P + tj[u]] = D[tj[u] * P + ti[u]] = nv[u];
      for (int t = lane; t < P * P; t += LANES) E[t] = red.Wt[t];
      __syncwarp();
    }
    red_invert<P, T>(D, lane);
  }
}

// in-place: rb (rhs) -> separator solution
template <int P, class T>
TDZ_DEV void red_solve(Red<T>& red, int nsep, int lane) {
  for (int s = 1; s < nsep; ++s) {  // y_s = b_s - F_s y_{s-1}
    cx<T> v = czero<T>();
    if (lane < P) {
      const cx<T>* F = red.E + s * P * P;
      v = red.rb[s * P + lane];
#pragma unroll
      for (int q = 0; q < P; ++q) v = cmsub(v, F[lane * P + q], red.rb[(s - 1) * P + q]);
    }
    __syncwarp();
    if (lane < P) red.rb[s * P + lane] = v;
    __syncwarp();
  }
  for (int s = nsep - 1; s >= 0; --s) {  // x_s = Pinv_s y_s - F_{s+1}^T x_{s+1}
    cx<T> v = czero<T>();
    if (lane < P) {
      const cx<T>* Pi = red.Dg + s * P * P;
#pragma unroll
      for (int q = 0; q < P; ++q) v = cmadd(v, Pi[lane * P + q], red.rb[s * P + q]);
      if (s + 1 < nsep) {
        const cx<T>* F = red.E + (s + 1) * P * P;
#pragma unroll
        for (int q = 0; q < P; ++q) v = cmsub(v, F[q * P + lane], red.rb[(s + 1) * P + q]);
      }
    }
    __syncwarp();
    if (lane < P) red.rb[s * P + lane] = v;
    __syncwarp();
  }
}

// ============================================================================ substitution
// Forward: g = L^-1 b' with b' = rhs - A(I, Sep_{k-1}) x_up, store g D^-1.
// Backward: x = L^-T (g D^-1) - (L_SI)^T x_dn, where L_SI are the multipliers sweep 1 stored for
// the lower separator rows (A_II^-1 A_IS = L^-T L_SI^T), so the lower coupling enters only here.
// The solution is accumulated in place: into the binary64 state (binary64 path) or into the
// double-float correction W (mixed path), for the interior and the lane's own separator rows.
template <class T, bool MIXED>
TDZ_DEV void accumulate(const RunDev& run, int idx, cx<T> x) {
  if constexpr (MIXED) {
    float4* W = run.W;
    const float4 q = W[idx];
    const ff wr = ff_addf(ff{q.x, q.z}, x.r), wi = ff_addf(ff{q.y, q.w}, x.i);
    W[idx] = make_float4(wr.h, wi.h, wr.l, wi.l);
  } else {
    double2* c = static_cast<double2*>(run.state);
    const double2 v = c[idx];
    c[idx] = make_double2(v.x + x.r, v.y + x.i);
  }
}

template <int P, class T, bool MIXED, bool CAP>
TDZ_DEV void substitute(const GeomDev& g, const RunDev& run, const Lane& L, T tau, T ebar, const Red<T>& red) {
  const int ks = L.ks;
  const int k = L.k;
  const cx<T>* __restrict__ rhs = static_cast<const cx<T>*>(run.rhs);
  const cx<T>* __restrict__ Lc = static_cast<const cx<T>*>(run.Lc);
  const cx<T>* __restrict__ Dv = static_cast<const cx<T>*>(run.Dv);
  cx<T>* __restrict__ gd = static_cast<cx<T>*>(run.gd);
  cx<T> xup[P], xdn[P];
#pragma unroll
  for (int j = 0; j < P; ++j) {
    xup[j] = L.up ? red.rb[(k - 1) * P + j] : czero<T>();
    xdn[j] = L.dn ? red.rb[k * P + j] : czero<T>();
  }
  cx<T> gw[P + 1];  // gw[d] = g_{i-d}
#pragma unroll
  for (int d = 0; d <= P; ++d) gw[d] = czero<T>();
  for (int i = 0; i < L.mI; ++i) {
    if (i + 4 < L.mI) {
      pf(rhs + ridx(i + 4, k, ks));
      pf(Dv + ridx(i + 4, k, ks));
#pragma unroll
      for (int d = 0; d < P; ++d) pf(Lc + ((i + 4) * P + d) * ks + k);
    }
    cx<T> b = rhs[ridx(i, k, ks)];
    if (L.up && i < P) {
#pragma unroll
      for (int j = 0; j < P; ++j)
        if (j >= i) b = cmsub(b, a_entry<P, T, MIXED, CAP>(g, bidx<P>(i, i + P - j, k, ks), tau, ebar), xup[j]);
    }
#pragma unroll
    for (int d = 1; d <= P; ++d)
      if (i - d >= 0) b = cmsub(b, Lc[((i - d) * P + d - 1) * ks + k], gw[d]);
#pragma unroll
    for (int d = P; d >= 2; --d) gw[d] = gw[d - 1];
    gw[1] = b;
    gd[ridx(i, k, ks)] = cmul(b, Dv[ridx(i, k, ks)]);
  }
  cx<T> xw[P + 1];  // xw[d] = x_{i+d}
#pragma unroll
  for (int d = 1; d <= P; ++d) xw[d] = xdn[d - 1];
  for (int i = L.mI - 1; i >= 0; --i) {
    if (i - 4 >= 0) {
      pf(gd + ridx(i - 4, k, ks));
      if constexpr (MIXED) pf(run.W + ridx(i - 4, k, ks));
      else pf(static_cast<const double2*>(run.state) + ridx(i - 4, k, ks));
#pragma unroll
      for (int d = 0; d < P; ++d) pf(Lc + ((i - 4) * P + d) * ks + k);
    }
    cx<T> x = gd[ridx(i, k, ks)];
#pragma unroll
    for (int d = 1; d <= P; ++d) x = cmsub(x, Lc[(i * P + d - 1) * ks + k], xw[d]);
#pragma unroll
    for (int d = P; d >= 2; --d) xw[d] = xw[d - 1];
    xw[1] = x;
    accumulate<T, MIXED>(run, ridx(i, k, ks), x);
  }
  if (L.dn) {
#pragma unroll
    for (int j = 0; j < P; ++j) accumulate<T, MIXED>(run, ridx(L.mI + j, k, ks), xdn[j]);
  }
}

// Second solve with the factors of the last factorisation (no refactorisation), in two lane phases
// that the caller separates with block barriers (neighbouring chunks may sit in different warps):
//   resolve_fwd: forward substitution with the stored L, which also eliminates into the lower
//                separator rows (their multipliers are stored too), giving that separator's rhs;
//   resolve_bwd: backward pass for the top of A_II^-1 r, whose product with the upper coupling
//                (-C^T z_T) is the upper separator's remaining rhs term;
// then the reduced solve with the stored block factors (red_solve) and substitute().
template <int P, class T, bool MIXED>
TDZ_DEV void resolve_fwd(const GeomDev& g, const RunDev& run, const Lane& L, Red<T>& red) {
  const int ks = L.ks;
  const int k = L.k;
  const cx<T>* __restrict__ rhs = static_cast<const cx<T>*>(run.rhs);
  const cx<T>* __restrict__ Lc = static_cast<const cx<T>*>(run.Lc);
  const cx<T>* __restrict__ Dv = static_cast<const cx<T>*>(run.Dv);
  cx<T>* __restrict__ gd = static_cast<cx<T>*>(run.gd);
  cx<T> sep[P];
#pragma unroll
  for (int j = 0; j < P; ++j) sep[j] = L.dn ? rhs[ridx(L.mI + j, k, ks)] : czero<T>();
  cx<T> gw[P + 1];
#pragma unroll
  for (int d = 0; d <= P; ++d) gw[d] = czero<T>();
  for (int i = 0; i < L.mI; ++i) {
    if (i + 4 < L.mI) {
      pf(rhs + ridx(i + 4, k, ks));
      pf(Dv + ridx(i + 4, k, ks));
#pragma unroll
      for (int d = 0; d < P; ++d) pf(Lc + ((i + 4) * P + d) * ks + k);
    }
    cx<T> b = rhs[ridx(i, k, ks)];
#pragma unroll
    for (int d = 1; d <= P; ++d)
      if (i - d >= 0) b = cmsub(b, Lc[((i - d) * P + d - 1) * ks + k], gw[d]);
#pragma unroll
    for (int d = P; d >= 2; --d) gw[d] = gw[d - 1];
    gw[1] = b;
    gd[ridx(i, k, ks)] = cmul(b, Dv[ridx(i, k, ks)]);
    if (L.dn && i >= L.mI - P) {
#pragma unroll
      for (int a = 1; a <= P; ++a) {
        const int j = i + a - L.mI;  // separator row index of row i+a
        if (j >= 0) sep[j] = cmsub(sep[j], Lc[(i * P + a - 1) * ks + k], b);
      }
    }
  }
  if (L.dn) {
#pragma unroll
    for (int j = 0; j < P; ++j) red.rb[k * P + j] = sep[j];
  }
}

template <int P, class T, bool MIXED, bool CAP>
TDZ_DEV void resolve_bwd(const GeomDev& g, const RunDev& run, const Lane& L, T tau, T ebar, Red<T>& red) {
  const int ks = L.ks;
  const int k = L.k;
  const cx<T>* __restrict__ Lc = static_cast<const cx<T>*>(run.Lc);
  const cx<T>* __restrict__ gd = static_cast<const cx<T>*>(run.gd);
  cx<T> zw[P + 1];  // zw[d] = z_{i+d}; the top P values end up in zw[1..P] reversed
#pragma unroll
  for (int d = 0; d <= P; ++d) zw[d] = czero<T>();
  for (int i = L.mI - 1; i >= 0; --i) {
    if (i - 4 >= 0) {
      pf(gd + ridx(i - 4, k, ks));
#pragma unroll
      for (int d = 0; d < P; ++d) pf(Lc + ((i - 4) * P + d) * ks + k);
    }
    cx<T> z = gd[ridx(i, k, ks)];
#pragma unroll
    for (int d = 1; d <= P; ++d) z = cmsub(z, Lc[(i * P + d - 1) * ks + k], zw[d]);
#pragma unroll
    for (int d = P; d >= 2; --d) zw[d] = zw[d - 1];
    zw[1] = z;
  }
  // zw[1 + i] = z_i for i = 0..P-1
#pragma unroll
  for (int j = 0; j < P; ++j) {
    cx<T> acc = czero<T>();
#pragma unroll
    for (int i = 0; i <= j; ++i)
      if (i < L.mI) acc = cmadd(acc, a_entry<P, T, MIXED, CAP>(g, bidx<P>(i, i + P - j, k, ks), tau, ebar), zw[1 + i]);
    red.rb[(k - 1) * P + j] = red.rb[(k - 1) * P + j] - acc;
  }
}

// ============================================================================ row helpers
// Location of local row j of lane k's chunk, possibly in a neighbouring chunk; false if none.
TDZ_DEV bool locate(const Lane& L, int j, int& row, int& chunk) {
  chunk = L.k;
  row = j;
  if (j < 0) {
    chunk = L.k - 1;
    row = j + L.m;
  } else if (j >= L.m) {
    chunk = L.k + 1;
    row = j - L.m;
  }
  return chunk >= 0 && chunk < L.K;
}

// ============================================================================ binary64 rhs
// r = -(tau W + i tau H_n) (2 c), scatter form over rows -P..m+P-1 with pending sums for P+1 rows (the
// absorbing layer's tau W only when CAP).
template <int P, bool CAP>
TDZ_DEV void rhs_fp64(const GeomDev& g, const RunDev& run, const Lane& L, double tau, double ebar) {
  const int ks = L.ks;
  const double2* c = static_cast<const double2*>(run.state);
  cx<double>* rhs = static_cast<cx<double>*>(run.rhs);
  cx<double> uw[P + 1];   // uw[d] = u_{j-d}
  cx<double> acc[P + 1];  // acc[d] = pending H u for row j-d
  cx<double> acw[P + 1];  // acw[d] = pending W u for row j-d (CAP)
#pragma unroll
  for (int d = 0; d <= P; ++d) {
    uw[d] = czero<double>();
    acc[d] = czero<double>();
    acw[d] = czero<double>();
  }
  for (int j = -P; j < L.m + P; ++j) {
    int row, chunk;
    const bool ok = locate(L, j, row, chunk);
    cx<double> u = czero<double>();
    double h[P + 1], wv[P + 1];
#pragma unroll
    for (int d = 0; d <= P; ++d) h[d] = wv[d] = 0.0;
    if (ok) {
      double2 cc = c[ridx(row, chunk, ks)];
      u = cx<double>{2.0 * cc.x, 2.0 * cc.y};
      if (j >= 0) {
#pragma unroll
        for (int d = 0; d <= P; ++d) {
          const int idx = bidx<P>(row, d, chunk, ks);
          h[d] = tau * fma(ebar, static_cast<const double*>(g.D)[idx], static_cast<const double*>(g.H)[idx]);
          if constexpr (CAP) wv[d] = tau * static_cast<const double*>(g.Wc)[idx];
        }
      }
    }
    // shift pending sums: acc[d] now refers to row j-d
#pragma unroll
    for (int d = P; d >= 1; --d) {
      acc[d] = acc[d - 1];
      if constexpr (CAP) acw[d] = acw[d - 1];
      uw[d] = uw[d - 1];
    }
    uw[0] = u;
    acc[0] = czero<double>();
    acw[0] = czero<double>();
    if (j >= 0 && j < L.m) {  // row j's own sum: lower part
#pragma unroll
      for (int d = 0; d <= P; ++d) {
        acc[0].r += h[d] * uw[d].r;
        acc[0].i += h[d] * uw[d].i;
        if constexpr (CAP) {
          acw[0].r += wv[d] * uw[d].r;
          acw[0].i += wv[d] * uw[d].i;
        }
      }
    }
    // upper contributions of row j to rows j-d
#pragma unroll
    for (int d = 1; d <= P; ++d) {
      if (j - d >= 0 && j - d < L.m) {
        acc[d].r += h[d] * u.r;
        acc[d].i += h[d] * u.i;
        if constexpr (CAP) {
          acw[d].r += wv[d] * u.r;
          acw[d].i += wv[d] * u.i;
        }
      }
    }
    const int jf = j - P;  // row complete
    if (jf >= 0 && jf < L.m) {
      // r = -i acc - acw  ->  (acc.i - acw.r, -acc.r - acw.i)
      rhs[ridx(jf, L.k, ks)] = cx<double>{acc[P].i - acw[P].r, -acc[P].r - acw[P].i};
    }
  }
}

// ============================================================================ double-float rhs
// r = -S w - (tau W + i tau H_n) u,  u = 2c + w (the absorbing layer's tau W only when CAP), all products
// in double-float (Dot2 accumulation), scatter
// form with pending sums for P+1 rows. Accumulates ||r||^2 and, when SCALE, ||S c||^2 (FP32) as the
// reference for the relative residual.
template <int P, bool SCALE, bool CAP>
TDZ_DEV void rhs_mixed(const GeomDev& g, const RunDev& run, const Lane& L, ff tau, ff ebar, float& rr, float& bb) {
  // complex double-float values are carried as packed pairs (real part in lane 0, imaginary in lane 1),
  // so each Dot2 step of the two components is one f32x2 instruction; the sums and their order are
  // those of the scalar form, component by component
  const int ks = L.ks;
  const float4* __restrict__ c = static_cast<const float4*>(run.state);
  const float4* __restrict__ W = run.W;
  const float4* __restrict__ A4 = static_cast<const float4*>(g.S);
  const float2* __restrict__ HD = static_cast<const float2*>(g.H);
  const float2* __restrict__ WC = static_cast<const float2*>(g.Wc);
  cx<float>* __restrict__ rhs = static_cast<cx<float>*>(run.rhs);
  const pcff zero = pcff{f2_pack(0.f, 0.f), f2_pack(0.f, 0.f)};
  pcff uw[P + 1], ww[P + 1];
  float2 cw[P + 1];
  pacc ac[P + 1];  // pending sums of rows j - d: (re, im)
  cx<float> sc[P + 1];
#pragma unroll
  for (int d = 0; d <= P; ++d) {
    uw[d] = zero;
    ww[d] = zero;
    cw[d] = make_float2(0.f, 0.f);
    pacc_zero(ac[d]);
    sc[d] = czero<float>();
  }
  rr = 0.f;
  bb = 0.f;
  for (int j = -P; j < L.m + P; ++j) {
    int row, chunk;
    const bool ok = locate(L, j, row, chunk);
    {
      int r2, c2;
      if (j + 2 < L.m + P && locate(L, j + 2, r2, c2)) {
        pf(c + ridx(r2, c2, ks));
        pf(W + ridx(r2, c2, ks));
        if (j + 2 >= 0) {
#pragma unroll
          for (int d = 0; d <= P; ++d) {
            pf(A4 + bidx<P>(r2, d, c2, ks));
            pf(HD + bidx<P>(r2, d, c2, ks));
          }
        }
      }
    }
    pcff u = zero, w = zero;
    float2 chi = make_float2(0.f, 0.f);
    ff s[P + 1], h[P + 1], wv[P + 1];
#pragma unroll
    for (int d = 0; d <= P; ++d) s[d] = h[d] = wv[d] = ff{0.f, 0.f};
    if (ok) {
      const float4 cc = c[ridx(row, chunk, ks)];  // (re.h, im.h, re.l, im.l)
      const float4 wq = W[ridx(row, chunk, ks)];
      w = pcff{f2_pack(wq.x, wq.y), f2_pack(wq.z, wq.w)};
      u = pcff_add(pcff{f2_pack(2.f * cc.x, 2.f * cc.y), f2_pack(2.f * cc.z, 2.f * cc.w)}, w);
      chi = make_float2(cc.x, cc.y);
      if (j >= 0) {
#pragma unroll
        for (int d = 0; d <= P; ++d) {
          const int idx = bidx<P>(row, d, chunk, ks);
          const float4 v = __ldg(A4 + idx);
          const float2 lo = __ldg(HD + idx);
          s[d] = ff{v.x, v.w};
          h[d] = ff_mul(tau, ff_add(ff{v.y, lo.x}, ff_mul(ebar, ff{v.z, lo.y})));  // tau (H0 + Ebar D)
          if constexpr (CAP) {
            const float2 wq2 = __ldg(WC + idx);
            wv[d] = ff_mul(tau, ff{wq2.x, wq2.y});  // tau W
          }
        }
      }
    }
#pragma unroll
    for (int d = P; d >= 1; --d) {
      ac[d] = ac[d - 1];
      uw[d] = uw[d - 1];
      ww[d] = ww[d - 1];
      if (SCALE) {
        sc[d] = sc[d - 1];
        cw[d] = cw[d - 1];
      }
    }
    uw[0] = u;
    ww[0] = w;
    cw[0] = chi;
    pacc_zero(ac[0]);
    sc[0] = czero<float>();
    // r.re = -S w.re + (tau H) u.im - (tau W) u.re ;  r.im = -S w.im - (tau H) u.re - (tau W) u.im
    // own row: four independent compensated partial sums (short dependency chains)
    if (j >= 0 && j < L.m) {
      pacc pa[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) pacc_zero(pa[q]);
#pragma unroll
      for (int d = 0; d <= P; ++d) {
        const pfac ns = pfac_of(-s[d].h, -s[d].l);
        pacc_mul(pa[(d & 1)], ns, ww[d]);
        pacc_mul(pa[2 + (d & 1)], pfac2_of(h[d].h, h[d].l, -h[d].h, -h[d].l), pcff_swap(uw[d]));
        if constexpr (CAP) pacc_mul(pa[(d & 1)], pfac_of(-wv[d].h, -wv[d].l), uw[d]);
        if (SCALE) {
          sc[0].r = fmaf(s[d].h, cw[d].x, sc[0].r);
          sc[0].i = fmaf(s[d].h, cw[d].y, sc[0].i);
        }
      }
      const pcff t = pcff_add(pcff_add(pacc_get(pa[0]), pacc_get(pa[1])), pcff_add(pacc_get(pa[2]), pacc_get(pa[3])));
      ac[0].s = t.h;
      ac[0].c = t.l;
    }
#pragma unroll
    for (int d = 1; d <= P; ++d) {
      if (j - d >= 0 && j - d < L.m) {
        pacc_mul(ac[d], pfac_of(-s[d].h, -s[d].l), w);
        pacc_mul(ac[d], pfac2_of(h[d].h, h[d].l, -h[d].h, -h[d].l), pcff_swap(u));
        if constexpr (CAP) pacc_mul(ac[d], pfac_of(-wv[d].h, -wv[d].l), u);
        if (SCALE) {
          sc[d].r = fmaf(s[d].h, chi.x, sc[d].r);
          sc[d].i = fmaf(s[d].h, chi.y, sc[d].i);
        }
      }
    }
    const int jf = j - P;
    if (jf >= 0 && jf < L.m) {
      const pcff a = pacc_get(ac[P]);
      const float2 f = f2_unpack(f2_add(a.h, a.l));  // ff_f on both lanes
      const cx<float> r = cx<float>{f.x, f.y};
      rhs[ridx(jf, L.k, ks)] = r;
      rr = fmaf(r.r, r.r, fmaf(r.i, r.i, rr));
      if (SCALE) bb = fmaf(sc[P].r, sc[P].r, fmaf(sc[P].i, sc[P].i, bb));
    }
  }
}

// ============================================================================ observables
// c^H M c = sum_j M_jj |c_j|^2 + 2 sum_{d>=1} M(j, j-d) Re(conj(c_j) c_{j-d}) for M = S, D, G, K.
template <int P>
TDZ_DEV void observe_fp64(const GeomDev& g, const RunDev& run, const Lane& L, bool cur, double out[5]) {
  const int ks = L.ks;
  const double2* c = static_cast<const double2*>(run.state);
  double2 cwin[P + 1];
#pragma unroll
  for (int d = 0; d <= P; ++d) cwin[d] = make_double2(0.0, 0.0);
  double s = 0, dd = 0, gg = 0, kk = 0, jv = 0;
  for (int j = -P; j < L.m; ++j) {
    int row, chunk;
    const bool ok = locate(L, j, row, chunk);
    const double2 cj = ok ? c[ridx(row, chunk, ks)] : make_double2(0.0, 0.0);
#pragma unroll
    for (int d = P; d >= 1; --d) cwin[d] = cwin[d - 1];
    cwin[0] = cj;
    if (j >= 0) {
#pragma unroll
      for (int d = 0; d <= P; ++d) {
        const double u = (d == 0 ? 1.0 : 2.0) * (cj.x * cwin[d].x + cj.y * cwin[d].y);
        const int idx = bidx<P>(row, d, chunk, ks);
        s = fma(static_cast<const double*>(g.S)[idx], u, s);
        dd = fma(static_cast<const double*>(g.D)[idx], u, dd);
        gg = fma(static_cast<const double*>(g.G)[idx], u, gg);
        kk = fma(static_cast<const double*>(g.Km)[idx], u, kk);
      }
      if (cur) {  // J = sum_{d >= 1} M(j, j-d) Im(conj(c_j) c_{j-d})
#pragma unroll
        for (int d = 1; d <= P; ++d)
          jv = fma(static_cast<const double*>(g.Mv)[bidx<P>(row, d, chunk, ks)], cj.x * cwin[d].y - cj.y * cwin[d].x, jv);
      }
    }
  }
  out[0] = s;
  out[1] = dd;
  out[2] = gg;
  out[3] = kk;
  out[4] = jv;
}

// Mixed path: c <- c + w (double-float), difference history d2 <- d1, d1 <- w, next predictor
// w <- 2 d1 - d2 (quadratic extrapolation, once two differences exist), and the observables of
// the new state, in one pass. The new values of the P rows above the chunk (the previous lane's
// separator) are formed from that lane's c and w before anyone overwrites them.
template <int P>
TDZ_DEV void update_observe_mixed(const GeomDev& g, const RunDev& run, const Lane& L, int hist_new, bool cur,
                                  double out[5]) {
  const int ks = L.ks;
  float4* __restrict__ c = static_cast<float4*>(run.state);
  float4* __restrict__ W = run.W;
  const float4* __restrict__ A4 = static_cast<const float4*>(g.S);
  const float2* __restrict__ HD = static_cast<const float2*>(g.H);
  const float4* __restrict__ GK = static_cast<const float4*>(g.G);
  cff cwin[P + 1];
#pragma unroll
  for (int d = 0; d <= P; ++d) cwin[d] = cff{{0.f, 0.f}, {0.f, 0.f}};
  if (L.active && L.up) {
#pragma unroll
    for (int q = 0; q < P; ++q) {  // row -P+q of chunk k-1 -> cwin[P-1-q] (the loop shifts before use)
      const int idx = ridx(L.m - P + q, L.k - 1, ks);
      const float4 cq = c[idx], wq = W[idx];
      cwin[P - 1 - q] = cff{ff_add(ff{cq.x, cq.z}, ff{wq.x, wq.z}), ff_add(ff{cq.y, cq.w}, ff{wq.y, wq.w})};
    }
  }
  __syncthreads();  // the previous chunk may belong to the other warp of this run: every thread calls this
  ffacc s, dd, gg, kk, jv;
  acc_zero(s);
  acc_zero(dd);
  acc_zero(gg);
  acc_zero(kk);
  acc_zero(jv);
  if (L.active) {
    for (int j = 0; j < L.m; ++j) {
      const int idx = ridx(j, L.k, ks);
      if (j + 2 < L.m) {
        const int i2 = ridx(j + 2, L.k, ks);
        pf(c + i2);
        pf(W + i2);
        pf(run.d1 + i2);
#pragma unroll
        for (int d = 0; d <= P; ++d) {
          pf(A4 + bidx<P>(j + 2, d, L.k, ks));
          pf(HD + bidx<P>(j + 2, d, L.k, ks));
          pf(GK + bidx<P>(j + 2, d, L.k, ks));
        }
      }
      const float4 cq = c[idx], wq = W[idx];
      const cff cj = cff{ff_add(ff{cq.x, cq.z}, ff{wq.x, wq.z}), ff_add(ff{cq.y, cq.w}, ff{wq.y, wq.w})};
      c[idx] = make_float4(cj.r.h, cj.i.h, cj.r.l, cj.i.l);
      const float2 n1 = make_float2(wq.x + wq.z, wq.y + wq.w);
      const float2 o1 = run.d1[idx];
      run.d2[idx] = o1;
      run.d1[idx] = n1;
      const float2 e = (hist_new >= 2) ? make_float2(2.f * n1.x - o1.x, 2.f * n1.y - o1.y) : make_float2(0.f, 0.f);
      W[idx] = make_float4(e.x, e.y, 0.f, 0.f);
#pragma unroll
      for (int d = P; d >= 1; --d) cwin[d] = cwin[d - 1];
      cwin[0] = cj;
      // per-row partial sums, two independent chains per matrix, folded into the lane totals once
      ffacc ps[2], pd[2], pg[2], pk[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        acc_zero(ps[q]);
        acc_zero(pd[q]);
        acc_zero(pg[q]);
        acc_zero(pk[q]);
      }
#pragma unroll
      for (int d = 0; d <= P; ++d) {
        ffacc ua;
        acc_zero(ua);
        acc_mul(ua, cj.r, cwin[d].r);
        acc_mul(ua, cj.i, cwin[d].i);
        ff u = acc_get(ua);
        if (d > 0) u = ff{2.f * u.h, 2.f * u.l};
        const int bi = bidx<P>(j, d, L.k, ks);
        const float4 v = __ldg(A4 + bi);
        const float2 lo = __ldg(HD + bi);
        const float4 gk = __ldg(GK + bi);
        acc_mul(ps[d & 1], ff{v.x, v.w}, u);
        acc_mul(pd[d & 1], ff{v.z, lo.y}, u);
        acc_mul(pg[d & 1], ff{gk.x, gk.y}, u);
        acc_mul(pk[d & 1], ff{gk.z, gk.w}, u);
      }
      acc_add(s, ff_add(acc_get(ps[0]), acc_get(ps[1])));
      acc_add(dd, ff_add(acc_get(pd[0]), acc_get(pd[1])));
      acc_add(gg, ff_add(acc_get(pg[0]), acc_get(pg[1])));
      acc_add(kk, ff_add(acc_get(pk[0]), acc_get(pk[1])));
      if (cur) {  // J = sum_{d >= 1} M(j, j-d) Im(conj(c_j) c_{j-d}), in double-float
        const float2* __restrict__ MV = static_cast<const float2*>(g.Mv);
#pragma unroll
        for (int d = 1; d <= P; ++d) {
          ffacc ui;
          acc_zero(ui);
          acc_mul(ui, cj.r, cwin[d].i);
          acc_mul(ui, ff_neg(cj.i), cwin[d].r);
          const float2 mq = __ldg(MV + bidx<P>(j, d, L.k, ks));
          acc_mul(jv, ff{mq.x, mq.y}, acc_get(ui));
        }
      }
    }
  }
  const ff fs = acc_get(s), fd = acc_get(dd), fg = acc_get(gg), fk = acc_get(kk), fj = acc_get(jv);
  out[0] = (double)fs.h + (double)fs.l;
  out[1] = (double)fd.h + (double)fd.l;
  out[2] = (double)fg.h + (double)fg.l;
  out[3] = (double)fk.h + (double)fk.l;
  out[4] = (double)fj.h + (double)fj.l;
}

// Sums over the K lanes of a run (consecutive threads of the block, possibly in several warps), the same
// value in every lane of the run, in a fixed order (lane 0 of the run adds its lanes' values in lane
// order). sh and tot are this block's per-lane scratch. Called by every thread of the block (it contains
// block barriers); threads without a run pass has = false.
template <int NV>
TDZ_DEV void run_sum(double (&v)[NV], double (*sh)[5], double (*tot)[5], int k, int K, bool has) {
  const int j = threadIdx.x;
#pragma unroll
  for (int q = 0; q < NV; ++q) sh[j][q] = v[q];
  __syncthreads();
  if (has && k == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = 0.0;
      for (int l = 0; l < K; ++l) t += sh[j + l][q];
      tot[j][q] = t;
    }
  }
  __syncthreads();
  if (has)
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = tot[j - k][q];
}


// The separator chains of a block's runs spread over its warps: chain j (the j-th run start in lane
// order) goes to warp j mod (warps per block), so two runs that start in one warp are not solved one
// after the other. Every thread of the block calls this (it holds a block barrier).
template <int P, class T>
TDZ_DEV void block_chains(const short* s_lead, int nlead, int* s_ns, int my_lead, bool lead, int nsep, bool go,
                          cx<T>* lane_area, cx<T>* wt, int wib, int nwarps, int lane, bool factor, bool solve) {
  if (lead) s_ns[my_lead] = go ? nsep : 0;
  __syncthreads();
  for (int j = wib; j < nlead; j += nwarps) {
    const int ns = s_ns[j];
    if (ns <= 0) continue;
    cx<T>* base = lane_area + (size_t)s_lead[j] * red_lane_elems(P);
    Red<T> r;
    r.Dg = base;
    r.E = base + ns * P * P;
    r.rb = base + 2 * ns * P * P;
    r.Wt = wt;
    if (factor) red_factor<P, T>(r, ns, lane);
    if (solve) red_solve<P, T>(r, ns, lane);
  }
}

// ============================================================================ the kernel
// A block takes a group of runs from a schedule built on the host: the group's lane map gives every thread
// its run and its lane (chunk) in that run, or no run. The block advances its runs in lock step: it
// crosses each phase of a step together (block barriers), so all warps of an SM execute the same code
// region at a time and the lanes of a run see each other's chunk boundaries and the run's shared reduced
// system. The adaptive refinement decides collectively how many extra solves the block makes; lanes whose
// run is already converged skip the work of those rounds.
template <int P, bool MIXED, bool CAP>
__global__ void __launch_bounds__(256) cn1d_kernel(StepArgs A) {
  using T = typename std::conditional<MIXED, float, double>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_group;
  __shared__ short s_lead[256];  // lanes that start a run, in lane order
  __shared__ int s_ns[256];      // their chain lengths for the current chain call
  __shared__ int s_wcnt[8];
  __shared__ int s_nlead;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int lpb = blockDim.x;
  cx<T>* lane_area = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* wt_area = lane_area + (size_t)lpb * red_lane_elems(P);
  double (*s_sum)[5] = reinterpret_cast<double (*)[5]>(wt_area + (size_t)(lpb / 32) * P * P);
  double (*s_tot)[5] = s_sum + lpb;

  while (true) {
    if (threadIdx.x == 0) s_group = atomicAdd(A.counter, 1);
    __syncthreads();
    const int grp = s_group;
    __syncthreads();
    if (grp >= A.ngroups) break;
    const int ent = A.lanes[(size_t)grp * lpb + threadIdx.x];
    const bool has = ent >= 0;
    const int rid = has ? (ent >> 8) : 0;
    RunDev run = A.runs[rid];
    const GeomDev g = A.geoms[run.geom];
    Lane L;
    L.k = has ? (ent & 255) : 0;
    L.K = has ? g.K : 1;
    L.m = g.m;
    L.ks = g.ks;
    L.active = has && L.k < g.K;
    L.up = L.active && L.k >= 1;
    L.dn = L.active && L.k < g.K - 1;
    L.mI = L.dn ? g.m - P : g.m;
    // the run's reduced system, in the shared memory of its own lanes (first lane at threadIdx.x - k)
    Red<T> red;
    {
      const int cap = L.K - 1;
      cx<T>* base = lane_area + (size_t)(threadIdx.x - L.k) * red_lane_elems(P);
      red.Dg = base;
      red.E = base + cap * P * P;
      red.rb = base + 2 * cap * P * P;
      red.Wt = wt_area + wib * P * P;
    }
    const bool lead = has && L.k == 0;  // writes the run's results; its warp runs the reduced system
    const unsigned starts = __ballot_sync(0xffffffffu, lead);
    int my_lead = -1;
    {
      if (lane == 0) s_wcnt[wib] = __popc(starts);
      __syncthreads();
      if (lead) {
        int off = __popc(starts & ((1u << lane) - 1u));
        for (int w = 0; w < wib; ++w) off += s_wcnt[w];
        my_lead = off;
        s_lead[off] = (short)threadIdx.x;
      }
      if (threadIdx.x == 0) {
        int n = 0;
        for (int w = 0; w < (lpb >> 5); ++w) n += s_wcnt[w];
        s_nlead = n;
      }
      __syncthreads();
    }
    const int nlead = s_nlead;
    const double* E = A.field + (size_t)rid * (A.nsteps + 1);
    double* obs = A.obs + (size_t)rid * A.nsteps * 5;
    int status = has ? run.status : TDZ_OK;
    double max_rel = 0.0;
    long long nsolve = 0;
    int hist = run.hist;
    for (long long s = 0; s < A.nsteps; ++s) {
      const bool work = has && status == TDZ_OK;
      Lane W = L;  // lanes of a warp whose run is finished or failed do no work this step
      W.active = L.active && work;
      W.up = W.active && L.up;
      W.dn = W.active && L.dn;
      const int nsep = work ? L.K - 1 : 0;
      const double ebar_d = 0.5 * (E[s] + E[s + 1]);
      const double tau_d = 0.5 * A.dt;
      double o[5] = {0, 0, 0, 0, 0};
      const bool cur = A.cur != nullptr;
      if constexpr (!MIXED) {
        if (W.active) rhs_fp64<P, CAP>(g, run, W, tau_d, ebar_d);
        __syncthreads();
        if (W.active) sweep1<P, double, false, CAP>(g, run, W, tau_d, ebar_d, red);
        __syncthreads();
        if (W.up) sweep2<P, double, false, CAP>(g, run, W, tau_d, ebar_d, red);
        __syncthreads();
        block_chains<P, double>(s_lead, nlead, s_ns, my_lead, lead, nsep, work, lane_area, red.Wt, wib, lpb >> 5, lane,
                                true, true);
        __syncthreads();
        if (W.active) substitute<P, double, false, CAP>(g, run, W, tau_d, ebar_d, red);  // c += delta
        __syncthreads();
        nsolve += work;
        if (W.active) observe_fp64<P>(g, run, W, cur, o);
      } else {
        const float tau_f = (float)tau_d, ebar_f = (float)ebar_d;
        const ff tau_ff = ff{tau_f, (float)(tau_d - (double)tau_f)};
        const ff ebar_ff = ff{ebar_f, (float)(ebar_d - (double)ebar_f)};
        // residual of the predictor y0 = c + w, then one factorising FP32 solve
        float rr = 0.f, bb = 0.f;
        if (W.active) rhs_mixed<P, true, CAP>(g, run, W, tau_ff, ebar_ff, rr, bb);
        double sums[2] = {(double)rr, (double)bb};
        run_sum(sums, s_sum, s_tot, L.k, L.K, has);
        const double bbs = fmax(sums[1], 1e-300);
        const double rel0 = sqrt(sums[0] / bbs);
        if (W.active) sweep1<P, float, true, CAP>(g, run, W, tau_f, ebar_f, red);
        __syncthreads();
        if (W.up) sweep2<P, float, true, CAP>(g, run, W, tau_f, ebar_f, red);
        __syncthreads();
        block_chains<P, float>(s_lead, nlead, s_ns, my_lead, lead, nsep, work, lane_area, red.Wt, wib, lpb >> 5, lane,
                               true, true);
        __syncthreads();
        if (W.active) substitute<P, float, true, CAP>(g, run, W, tau_f, ebar_f, red);  // w += delta
        __syncthreads();
        nsolve += work;
        // residual after the solve; refine with the stored factors while above tolerance
        if (W.active) rhs_mixed<P, false, CAP>(g, run, W, tau_ff, ebar_ff, rr, bb);
        double r1[1] = {W.active ? (double)rr : 0.0};
        run_sum(r1, s_sum, s_tot, L.k, L.K, has);
        double rel = sqrt(r1[0] / bbs);
        const double rho = fmin(rel / fmax(rel0, 1e-300), 1.0);  // contraction of one FP32 solve
        int it = 1;
        bool ok = !work || rel <= A.tol;
        bool need = !ok && it < A.max_it;
        while (__syncthreads_or(need)) {
          if (need && W.active) resolve_fwd<P, float, true>(g, run, W, red);
          __syncthreads();
          if (need && W.up) resolve_bwd<P, float, true, CAP>(g, run, W, tau_f, ebar_f, red);
          __syncthreads();
          block_chains<P, float>(s_lead, nlead, s_ns, my_lead, lead, nsep, need, lane_area, red.Wt, wib, lpb >> 5,
                                 lane, false, true);
          __syncthreads();
          if (need && W.active) substitute<P, float, true, CAP>(g, run, W, tau_f, ebar_f, red);
          __syncthreads();
          if (need) {
            nsolve++;
            ++it;
            const double predicted = rho * rel;
            if (predicted <= 0.1 * A.tol && rho < 1e-2) {  // contraction certain: accept unchecked
              rel = predicted;
              ok = true;
            }
          }
          const bool check = need && !ok;
          if (check && W.active) rhs_mixed<P, false, CAP>(g, run, W, tau_ff, ebar_ff, rr, bb);
          double rc[1] = {(check && W.active) ? (double)rr : 0.0};
          run_sum(rc, s_sum, s_tot, L.k, L.K, has);
          if (check) {
            rel = sqrt(rc[0] / bbs);
            ok = rel <= A.tol;
          }
          need = need && !ok && it < A.max_it;
        }
        if (work) {
          max_rel = fmax(max_rel, rel);
          if (!ok && status == TDZ_OK) status = TDZ_ENOCONV;
          hist = hist + 1;
        }
        __syncthreads();
        update_observe_mixed<P>(g, run, W, hist, cur, o);
      }
      run_sum(o, s_sum, s_tot, L.k, L.K, has);
      if (work) {
        const double Et = E[s + 1];
        if (lead) {
          double* row = obs + s * 5;
          row[0] = (double)(A.step0 + s + 1) * A.dt;
          row[1] = Et;
          row[2] = o[1];
          row[3] = -o[2] - Et * o[3];
          row[4] = o[0];
          if (cur) A.cur[(size_t)rid * A.nsteps + s] = o[4];
        }
        if (!isfinite(o[0]) || !isfinite(o[1])) status = TDZ_ENONFINITE;
      }
      __syncthreads();
    }
    if (lead) {
      A.runs[rid].status = status;
      A.runs[rid].hist = hist;
      A.runs[rid].max_rel = fmax(run.max_rel, max_rel);
      A.runs[rid].nsolve = run.nsolve + nsolve;
    }
    __syncthreads();
  }
}

}  // namespace tdz

// ============================================================================ batched state upload
// All runs' coefficients, natural order, concatenated in run order (re, im interleaved) -> each run's
// chunk-interleaved state; padding rows zero; the mixed path's correction and difference history
// are reset (like a per-run set_state). One block per run. *bad is set on a non-finite coefficient.
template <bool MIXED>
__global__ void k_set_states(const double* __restrict__ src, const long long* __restrict__ off, tdz::RunDev* runs,
                             const tdz::GeomDev* __restrict__ geoms, int nruns, int* bad) {
  for (int r = blockIdx.x; r < nruns; r += gridDim.x) {
    const tdz::RunDev R = runs[r];
    const tdz::GeomDev g = geoms[R.geom];
    const long long base = off[r];
    const long long rows = (long long)g.m * g.ks;
    for (long long e = threadIdx.x; e < rows; e += blockDim.x) {
      const int i = (int)(e / g.ks), k = (int)(e % g.ks);
      const long long gi = (long long)k * g.m + i;
      double re = 0.0, im = 0.0;
      if (k < g.K && gi < g.n) {
        re = src[2 * (base + gi)];
        im = src[2 * (base + gi) + 1];
        if (!isfinite(re) || !isfinite(im)) *bad = 1;
      }
      if constexpr (MIXED) {
        const float rh = (float)re, ih = (float)im;
        static_cast<float4*>(R.state)[e] = make_float4(rh, ih, (float)(re - (double)rh), (float)(im - (double)ih));
        R.W[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        R.d1[e] = make_float2(0.f, 0.f);
        R.d2[e] = make_float2(0.f, 0.f);
      } else {
        static_cast<double2*>(R.state)[e] = make_double2(re, im);
      }
    }
    if (threadIdx.x == 0) {
      runs[r].status = TDZ_OK;
      runs[r].hist = 0;
    }
  }
}

// ============================================================================ host side
using namespace tdz;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return TDZ_ECUDA;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Dynamic shared memory of a block of `lanes` threads (the layout is described at red_lane_elems).
size_t block_smem(int P, bool mixed, int lanes) {
  const size_t cxsz = mixed ? 8 : 16;
  return (size_t)lanes * red_lane_elems(P) * cxsz + (size_t)(lanes / 32) * P * P * cxsz +
         (size_t)lanes * 10 * sizeof(double);
}

// Most warps (<= 8) a block can have within `maxsm` bytes of shared memory.
int max_warps(int P, bool mixed, int maxsm) {
  int w = 8;
  while (w > 1 && block_smem(P, mixed, 32 * w) > (size_t)maxsm) --w;
  return w;
}

// The dynamic shared-memory limit of a kernel is one attribute of the function, shared by every host
// thread that launches it. It is only ever raised, straight to the largest size any launch of this
// instantiation can use on the device (a block of the most warps its shared memory allows), so a launch
// made on one thread never finds the limit lowered by a call on another.
template <int P, bool M, bool CAP>
cudaError_t ensure_smem(size_t need) {
  static std::mutex mu;
  static size_t set_to[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (set_to[dev] >= need) return cudaSuccess;
  int maxsm = 0;
  e = cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const size_t cap = block_smem(P, M, 32 * max_warps(P, M, maxsm));
  const size_t v = std::max(need, cap);
  e = cudaFuncSetAttribute(cn1d_kernel<P, M, CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v);
  if (e == cudaSuccess) set_to[dev] = v;
  return e;
}

}  // namespace

namespace {

// Chunks (lanes) of a run of n rows for a target of mt rows per lane: K = ceil(n / mt), at most `lanes`,
// reduced until every interior is at least P + 1 rows long (the separator of a chunk is its last P rows).
int chunks_for(int n, int P, int mt, int lanes) {
  int K = std::max(1, std::min(lanes, (n + mt - 1) / mt));
  int m = (n + K - 1) / K;
  while (K > 1 && m - P < P + 1) {
    --K;
    m = (n + K - 1) / K;
  }
  return K;
}

// Schedule of the persistent launch: the runs are packed lane by lane into groups of `lpb` lanes (one block
// each). Every geometry gets the K chunks that give its runs about the same rows per lane, mt, so that all
// lanes of the launch take about the same time per step; the runs then go, largest K first and the runs of
// one geometry together (they share their band arrays), into the first group with room (first-fit
// decreasing). mt starts at the batch's rows over all resident lanes and grows until the groups fit the
// resident blocks (one round); a batch with more runs than resident lanes runs its groups in several
// rounds. Returns the lane map (groups x lpb; run << 8 | lane of the run, or -1) and each geometry's K.
struct Packing {
  std::vector<int> lanes;
  int ngroups = 0;
  std::vector<int> gK;
};

Packing pack_runs(const std::vector<int>& gsize, const int* ops_index, int nruns, int P, int lpb, int resident) {
  const int nops = (int)gsize.size();
  long long total = 0;
  int nmax = 1;
  for (int r = 0; r < nruns; ++r) total += gsize[ops_index[r]];
  for (int g = 0; g < nops; ++g) nmax = std::max(nmax, gsize[g]);
  const long long slots = (long long)std::max(1, resident) * lpb;
  int mt = std::max(2 * P + 1, (int)((total + slots - 1) / slots));
  Packing pk;
  std::vector<int> order(nruns);
  for (;;) {
    std::vector<int> gK(nops);
    for (int g = 0; g < nops; ++g) gK[g] = chunks_for(gsize[g], P, mt, lpb);
    for (int r = 0; r < nruns; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      const int kx = gK[ops_index[x]], ky = gK[ops_index[y]];
      return kx != ky ? kx > ky : ops_index[x] < ops_index[y];
    });
    std::vector<int> fill;
    std::vector<std::vector<int>> members;
    for (int r : order) {
      const int K = gK[ops_index[r]];
      size_t b = 0;
      while (b < fill.size() && fill[b] + K > lpb) ++b;
      if (b == fill.size()) {
        fill.push_back(0);
        members.emplace_back();
      }
      fill[b] += K;
      members[b].push_back(r);
    }
    if ((int)fill.size() <= resident || mt >= nmax) {
      pk.gK = gK;
      pk.ngroups = (int)fill.size();
      pk.lanes.assign((size_t)pk.ngroups * lpb, -1);
      for (int b = 0; b < pk.ngroups; ++b) {
        int j = 0;
        for (int r : members[b])
          for (int k = 0; k < gK[ops_index[r]]; ++k) pk.lanes[(size_t)b * lpb + j++] = (r << 8) | k;
      }
      return pk;
    }
    mt += std::max(1, mt / 32);
  }
}

}  // namespace

struct tdz_batch {
  tdz::NdBatch* nd = nullptr;  // 2-D / 3-D batches are served by tdz_nd.cu
  int prec = TDZ_FP64;
  int P = 0;
  int nruns = 0;
  cudaStream_t stream = nullptr;
  struct G {
    int n, m, K, ks;  // size, rows per chunk, chunks, interleave stride (32 x warps per run)
  };
  std::vector<G> geo;
  std::vector<int> run_geom;
  std::vector<DevBuf> bufs;  // everything allocated, freed in destroy
  GeomDev* d_geoms = nullptr;
  RunDev* d_runs = nullptr;
  std::vector<RunDev> h_runs;
  int* d_lanes = nullptr;  // lane map of the launch's groups (pack_runs)
  long long* d_off = nullptr;  // first coefficient of every run in a concatenated state vector
  std::vector<long long> h_off;
  double* d_stage = nullptr;   // staging for a host-side concatenated state (allocated on first use)
  int* d_bad = nullptr;
  int ngroups = 0;
  int* d_counter = nullptr;
  double* d_obs = nullptr;
  size_t obs_steps = 0;
  double* d_field = nullptr;
  size_t field_len = 0;
  long long last_nsteps = 0;
  int64_t total_dof = 0;
  size_t dev_bytes = 0;
  int lanes_per_block = 256;
  int blocks = 0;
  bool cap = false;  // some geometry has an absorbing layer: every run takes the kernel with the W band
  // total dipole velocity per step (TDZ_OPT_CURRENT): velocity bands uploaded on first use, per-step buffer
  bool current = false;
  std::vector<GeomDev> h_geoms;
  std::vector<const Ops*> ops_of;
  double* d_cur = nullptr;
  size_t cur_len = 0;
  double tol = 1e-11;
  int max_it = 6;

  void* alloc(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    cudaMemsetAsync(p, 0, bytes, stream);
    bufs.push_back({p, bytes});
    dev_bytes += bytes;
    return p;
  }
  ~tdz_batch() {
    if (nd) tdz::nd_batch_destroy(nd);
    for (auto& b : bufs) cudaFree(b.p);
    if (d_obs) cudaFree(d_obs);
    if (d_field) cudaFree(d_field);
    if (d_stage) cudaFree(d_stage);
    if (d_cur) cudaFree(d_cur);
  }
};

namespace {

template <int P, bool M, bool CAP>
cudaError_t launch_p(tdz_batch* b, const StepArgs& a) {
  const size_t sm = block_smem(P, M, b->lanes_per_block);
  cudaError_t e = ensure_smem<P, M, CAP>(sm);
  if (e != cudaSuccess) return e;
  cn1d_kernel<P, M, CAP><<<b->blocks, b->lanes_per_block, sm, b->stream>>>(a);
  return cudaGetLastError();
}

template <bool M, bool CAP>
cudaError_t launch_c(tdz_batch* b, const StepArgs& a) {
  switch (b->P) {
    case 1: return launch_p<1, M, CAP>(b, a);
    case 2: return launch_p<2, M, CAP>(b, a);
    case 3: return launch_p<3, M, CAP>(b, a);
    case 4: return launch_p<4, M, CAP>(b, a);
    case 5: return launch_p<5, M, CAP>(b, a);
    case 6: return launch_p<6, M, CAP>(b, a);
    case 7: return launch_p<7, M, CAP>(b, a);
    case 8: return launch_p<8, M, CAP>(b, a);
  }
  return cudaErrorInvalidValue;
}

template <bool M>
cudaError_t launch(tdz_batch* b, const StepArgs& a) {
  return b->cap ? launch_c<M, true>(b, a) : launch_c<M, false>(b, a);
}

}  // namespace

extern "C" {

int tdz_batch_create(const tdz_ops* const* ops, int nops, int nruns, const int* ops_index, int precision,
                     void* cuda_stream, tdz_batch** out) {
  if (!ops || nops < 1 || nruns < 1 || !ops_index || !out) return TDZ_EINVAL;
  if (precision != TDZ_FP64 && precision != TDZ_MIXED) return TDZ_EINVAL;
  for (int g = 0; g < nops; ++g)
    if (!ops[g]) return TDZ_EINVAL;
  for (int r = 0; r < nruns; ++r)
    if (ops_index[r] < 0 || ops_index[r] >= nops) return TDZ_EINVAL;
  if (ops[0]->o.dim > 1) {
    tdz_batch* b = new (std::nothrow) tdz_batch;
    if (!b) return TDZ_ENOMEM;
    b->prec = precision;
    b->nruns = nruns;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    const int rc = tdz::nd_batch_create(ops, nops, nruns, ops_index, precision, cuda_stream, &b->nd);
    if (rc != TDZ_OK) {
      delete b;
      return rc;
    }
    for (int r = 0; r < nruns; ++r) b->total_dof += tdz::nd_run_size(b->nd, r);
    b->dev_bytes = tdz::nd_device_bytes(b->nd);
    *out = b;
    return TDZ_OK;
  }
  for (int g = 0; g < nops; ++g) {
    if (ops[g]->o.dim != 1) {
      set_error("tdz_batch_create: all operators of a batch must have the same dimension");
      return TDZ_EUNSUPPORTED;
    }
    if (ops[g]->o.n[0] < ops[g]->o.p[0] + 1) {
      set_error("tdz_batch_create: a run needs at least degree+1 coefficients");
      return TDZ_EINVAL;
    }
    if (ops[g]->o.p[0] != ops[0]->o.p[0]) {
      set_error("tdz_batch_create: all operators of a batch must have the same degree");
      return TDZ_EUNSUPPORTED;
    }
  }
  for (int r = 0; r < nruns; ++r)
    if (ops_index[r] < 0 || ops_index[r] >= nops) return TDZ_EINVAL;
  const int P = ops[0]->o.p[0];
  if (P < 1 || P > MAXP) return TDZ_EUNSUPPORTED;
  tdz_batch* b = new (std::nothrow) tdz_batch;
  if (!b) return TDZ_ENOMEM;
  b->prec = precision;
  b->P = P;
  for (int g = 0; g < nops; ++g) b->cap = b->cap || ops[g]->o.has_cap();
  b->nruns = nruns;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  const bool mixed = precision == TDZ_MIXED;
  const int P1 = P + 1;
  const size_t Tsz = mixed ? 8 : 16;  // complex element of the solve precision
  // ---------------------------------------------------------------- launch shape and schedule
  int dev = 0, sms = 148, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // blocks resident per SM: shared memory (228 KB per SM, 1 KB reserved per block) and registers (the
  // kernels are built for at most 255 per thread)
  auto resident_per_sm = [&](int lanes) {
    return std::max(1, std::min((int)((size_t)228 * 1024 / (block_smem(P, mixed, lanes) + 1024)),
                                65536 / (256 * lanes)));
  };
  const int lpb = 32 * max_warps(P, mixed, maxsm);
  const int per_sm = resident_per_sm(lpb);
  std::vector<int> gsize(nops);
  for (int gi = 0; gi < nops; ++gi) gsize[gi] = (int)ops[gi]->o.n[0];
  const Packing pk = pack_runs(gsize, ops_index, nruns, P, lpb, sms * per_sm);

  // ---------------------------------------------------------------- geometries
  std::vector<GeomDev> hg(nops);
  b->geo.resize(nops);
  for (int gi = 0; gi < nops; ++gi) {
    const Ops& o = ops[gi]->o;
    const int n = (int)o.n[0];
    const int K = pk.gK[gi], m = (n + K - 1) / K, LS = K;
    b->geo[gi] = {n, m, K, LS};
    const size_t nb = (size_t)m * P1 * LS;
    const Band* src[6] = {&o.S, &o.H0, &o.D, &o.G, &o.K, &o.W};
    // value of matrix q at interleaved position (i, d, k); padding rows are identity in S
    auto val = [&](int q, int i, int d, int k) -> double {
      const int64_t gr = (int64_t)k * m + i;
      if (k >= K) return 0.0;
      if (gr < n) return (gr - d >= 0) ? src[q]->at(gr, d) : 0.0;
      return (q == 0 && d == 0) ? 1.0 : 0.0;
    };
    auto hi = [](double v) { return (float)v; };
    auto lo = [](double v) { return (float)(v - (double)(float)v); };
    void* dst[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    auto val_w = [&](int i, int d, int k) -> double { return o.has_cap() ? val(5, i, d, k) : 0.0; };
    auto upload = [&](const void* h, size_t bytes) -> void* {
      void* p = b->alloc(bytes);
      if (!p) return nullptr;
      if (cudaMemcpyAsync(p, h, bytes, cudaMemcpyHostToDevice, b->stream) != cudaSuccess) return nullptr;
      if (cudaStreamSynchronize(b->stream) != cudaSuccess) return nullptr;
      return p;
    };
    if (mixed) {
      std::vector<float> a4(nb * 4), hd(nb * 2), gk(nb * 4);
      for (int k = 0; k < LS; ++k)
        for (int i = 0; i < m; ++i)
          for (int d = 0; d <= P; ++d) {
            const size_t idx = ((size_t)i * P1 + d) * LS + k;
            const double S = val(0, i, d, k), H = val(1, i, d, k), D = val(2, i, d, k), Gv = val(3, i, d, k),
                         Kv = val(4, i, d, k);
            a4[4 * idx + 0] = hi(S);
            a4[4 * idx + 1] = hi(H);
            a4[4 * idx + 2] = hi(D);
            a4[4 * idx + 3] = lo(S);
            hd[2 * idx + 0] = lo(H);
            hd[2 * idx + 1] = lo(D);
            gk[4 * idx + 0] = hi(Gv);
            gk[4 * idx + 1] = lo(Gv);
            gk[4 * idx + 2] = hi(Kv);
            gk[4 * idx + 3] = lo(Kv);
          }
      dst[0] = upload(a4.data(), nb * 16);
      dst[1] = upload(hd.data(), nb * 8);
      dst[3] = upload(gk.data(), nb * 16);
      if (b->cap) {
        std::vector<float> wc(nb * 2);
        for (int k = 0; k < LS; ++k)
          for (int i = 0; i < m; ++i)
            for (int d = 0; d <= P; ++d) {
              const size_t idx = ((size_t)i * P1 + d) * LS + k;
              wc[2 * idx + 0] = hi(val_w(i, d, k));
              wc[2 * idx + 1] = lo(val_w(i, d, k));
            }
        dst[5] = upload(wc.data(), nb * 8);
        if (!dst[5]) dst[0] = nullptr;
      }
      if (!dst[0] || !dst[1] || !dst[3]) {
        delete b;
        set_error("tdz_batch_create: band upload failed");
        return TDZ_ENOMEM;
      }
    } else {
      std::vector<double> hd(nb);
      for (int q = 0; q < (b->cap ? 6 : 5); ++q) {
        for (int k = 0; k < LS; ++k)
          for (int i = 0; i < m; ++i)
            for (int d = 0; d <= P; ++d)
              hd[((size_t)i * P1 + d) * LS + k] = q == 5 ? val_w(i, d, k) : val(q, i, d, k);
        dst[q] = upload(hd.data(), nb * 8);
        if (!dst[q]) {
          delete b;
          set_error("tdz_batch_create: band upload failed");
          return TDZ_ENOMEM;
        }
      }
    }
    hg[gi] = GeomDev{n, m, K, LS, dst[0], dst[1], dst[2], dst[3], dst[4], b->cap ? dst[5] : nullptr, nullptr};
  }
  // ---------------------------------------------------------------- runs
  b->h_runs.resize(nruns);
  b->run_geom.assign(ops_index, ops_index + nruns);
  for (int r = 0; r < nruns; ++r) {
    const auto& G = b->geo[ops_index[r]];
    const size_t rows = (size_t)G.m * G.ks;
    RunDev R{};
    R.geom = ops_index[r];
    R.status = TDZ_OK;
    R.hist = 0;
    R.state = b->alloc(rows * 16);
    R.rhs = b->alloc(rows * Tsz);
    R.Lc = b->alloc(rows * P * Tsz);
    R.Dv = b->alloc(rows * Tsz);
    R.gd = b->alloc(rows * Tsz);
    R.dl = b->alloc(rows * Tsz);
    if (mixed) {
      R.d1 = static_cast<float2*>(b->alloc(rows * 8));
      R.d2 = static_cast<float2*>(b->alloc(rows * 8));
      R.W = static_cast<float4*>(b->alloc(rows * 16));
    }
    if (!R.state || !R.rhs || !R.Lc || !R.Dv || !R.gd || !R.dl || (mixed && (!R.d1 || !R.d2 || !R.W))) {
      delete b;
      return TDZ_ENOMEM;
    }
    b->h_runs[r] = R;
    b->total_dof += G.n;
  }
  b->d_geoms = static_cast<GeomDev*>(b->alloc(sizeof(GeomDev) * nops));
  b->d_runs = static_cast<RunDev*>(b->alloc(sizeof(RunDev) * nruns));
  b->ngroups = pk.ngroups;
  b->d_lanes = static_cast<int*>(b->alloc(sizeof(int) * pk.lanes.size()));
  b->d_counter = static_cast<int*>(b->alloc(sizeof(int)));
  b->d_off = static_cast<long long*>(b->alloc(sizeof(long long) * (nruns + 1)));
  b->d_bad = static_cast<int*>(b->alloc(sizeof(int)));
  b->h_off.assign(nruns + 1, 0);
  for (int r = 0; r < nruns; ++r) b->h_off[r + 1] = b->h_off[r] + b->geo[ops_index[r]].n;
  if (!b->d_geoms || !b->d_runs || !b->d_lanes || !b->d_counter || !b->d_off || !b->d_bad) {
    delete b;
    return TDZ_ENOMEM;
  }
  cudaMemcpyAsync(b->d_geoms, hg.data(), sizeof(GeomDev) * nops, cudaMemcpyHostToDevice, b->stream);
  b->h_geoms = hg;
  for (int g = 0; g < nops; ++g) b->ops_of.push_back(&ops[g]->o);
  cudaMemcpyAsync(b->d_runs, b->h_runs.data(), sizeof(RunDev) * nruns, cudaMemcpyHostToDevice, b->stream);
  cudaMemcpyAsync(b->d_lanes, pk.lanes.data(), sizeof(int) * pk.lanes.size(), cudaMemcpyHostToDevice, b->stream);
  cudaMemcpyAsync(b->d_off, b->h_off.data(), sizeof(long long) * (nruns + 1), cudaMemcpyHostToDevice, b->stream);
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "tdz_batch_create");
  }
  b->lanes_per_block = lpb;
  b->blocks = std::max(1, std::min(b->ngroups, sms * per_sm));
  *out = b;
  return TDZ_OK;
}

int tdz_batch_set_refinement(tdz_batch* b, double tol, int max_solves) {
  if (!b || !(tol > 0) || max_solves < 1 || max_solves > 64) return TDZ_EINVAL;
  if (b->nd) tdz::nd_set_refinement(b->nd, tol, max_solves);
  b->tol = tol;
  b->max_it = max_solves;
  return TDZ_OK;
}

int tdz_batch_info(const tdz_batch* b, int* nruns, int64_t* total_dof, size_t* device_bytes) {
  if (!b) return TDZ_EINVAL;
  if (nruns) *nruns = b->nruns;
  if (total_dof) *total_dof = b->total_dof;
  if (device_bytes) *device_bytes = b->dev_bytes;
  return TDZ_OK;
}

int tdz_set_state(tdz_batch* b, int run, const double* c) {
  if (!b || !c || run < 0 || run >= b->nruns) return TDZ_EINVAL;
  if (b->nd) return tdz::nd_set_state(b->nd, run, c, is_device_ptr(c));
  const auto& G = b->geo[b->run_geom[run]];
  const int n = G.n, m = G.m, LS = G.ks;
  std::vector<double> hc((size_t)2 * n);
  cudaError_t e;
  if (is_device_ptr(c)) {
    e = cudaMemcpyAsync(hc.data(), c, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tdz_set_state");
  } else {
    std::memcpy(hc.data(), c, sizeof(double) * 2 * n);
  }
  for (int i = 0; i < 2 * n; ++i)
    if (!std::isfinite(hc[i])) {
      set_error("tdz_set_state: non-finite coefficient");
      return TDZ_ENONFINITE;
    }
  const size_t rows = (size_t)m * LS;
  RunDev& R = b->h_runs[run];
  if (b->prec == TDZ_MIXED) {
    std::vector<float> s(rows * 4, 0.f);
    for (int g = 0; g < n; ++g) {
      const size_t idx = (size_t)(g % m) * LS + g / m;
      const double re = hc[2 * g], im = hc[2 * g + 1];
      const float rh = (float)re, ih = (float)im;
      s[4 * idx + 0] = rh;
      s[4 * idx + 1] = ih;
      s[4 * idx + 2] = (float)(re - (double)rh);
      s[4 * idx + 3] = (float)(im - (double)ih);
    }
    e = cudaMemcpyAsync(R.state, s.data(), rows * 16, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(R.d1, 0, rows * 8, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(R.d2, 0, rows * 8, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(R.W, 0, rows * 16, b->stream);
  } else {
    std::vector<double> s(rows * 2, 0.0);
    for (int g = 0; g < n; ++g) {
      const size_t idx = (size_t)(g % m) * LS + g / m;
      s[2 * idx] = hc[2 * g];
      s[2 * idx + 1] = hc[2 * g + 1];
    }
    e = cudaMemcpyAsync(R.state, s.data(), rows * 16, cudaMemcpyHostToDevice, b->stream);
  }
  // reset history and status of this run
  if (e == cudaSuccess) {
    RunDev upd = R;
    upd.hist = 0;
    upd.status = TDZ_OK;
    e = cudaMemcpyAsync(&b->d_runs[run].status, &upd.status, sizeof(int) * 2, cudaMemcpyHostToDevice, b->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tdz_set_state");
  return TDZ_OK;
}

int tdz_get_state(const tdz_batch* b, int run, double* c) {
  if (!b || !c || run < 0 || run >= b->nruns) return TDZ_EINVAL;
  if (b->nd) return tdz::nd_get_state(b->nd, run, c, is_device_ptr(c));
  const auto& G = b->geo[b->run_geom[run]];
  const int n = G.n, m = G.m, LS = G.ks;
  const size_t rows = (size_t)m * LS;
  const RunDev& R = b->h_runs[run];
  std::vector<double> hc((size_t)2 * n);
  cudaError_t e;
  if (b->prec == TDZ_MIXED) {
    std::vector<float> s(rows * 4);
    e = cudaMemcpyAsync(s.data(), R.state, rows * 16, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tdz_get_state");
    for (int g = 0; g < n; ++g) {
      const size_t idx = (size_t)(g % m) * LS + g / m;
      hc[2 * g] = (double)s[4 * idx] + (double)s[4 * idx + 2];
      hc[2 * g + 1] = (double)s[4 * idx + 1] + (double)s[4 * idx + 3];
    }
  } else {
    std::vector<double> s(rows * 2);
    e = cudaMemcpyAsync(s.data(), R.state, rows * 16, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tdz_get_state");
    for (int g = 0; g < n; ++g) {
      const size_t idx = (size_t)(g % m) * LS + g / m;
      hc[2 * g] = s[2 * idx];
      hc[2 * g + 1] = s[2 * idx + 1];
    }
  }
  if (is_device_ptr(c)) {
    e = cudaMemcpyAsync(c, hc.data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tdz_get_state");
  } else {
    std::memcpy(c, hc.data(), sizeof(double) * 2 * n);
  }
  return TDZ_OK;
}

int tdz_propagate(tdz_batch* b, const double* field, double dt, int64_t step0, int64_t nsteps) {
  if (!b || !field || nsteps < 1 || step0 < 0 || !(dt > 0) || !std::isfinite(dt)) return TDZ_EINVAL;
  if (b->nd) {
    // the 2-D/3-D driver reads the field samples on the host
    const size_t cnt = (size_t)b->nruns * (nsteps + 1);
    std::vector<double> hf;
    const double* fh = field;
    const int D = tdz::nd_dim(b->nd);
    if (is_device_ptr(field)) {
      hf.resize(cnt * D);
      cudaError_t e = cudaMemcpy(hf.data(), field, sizeof(double) * cnt * D, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "tdz_propagate: field download");
      fh = hf.data();
    }
    for (size_t k = 0; k < cnt * D; ++k)
      if (!std::isfinite(fh[k])) {
        set_error("tdz_propagate: non-finite field sample");
        return TDZ_ENONFINITE;
      }
    const int rc = tdz::nd_propagate(b->nd, fh, dt, step0, nsteps);
    b->last_nsteps = nsteps;
    return rc;
  }
  const size_t need = (size_t)b->nruns * (nsteps + 1);
  const double* dfield = field;
  cudaError_t e;
  if (!is_device_ptr(field)) {
    if (b->field_len < need) {
      if (b->d_field) cudaFreeAsync(b->d_field, b->stream);
      b->d_field = nullptr;
      e = cudaMallocAsync(reinterpret_cast<void**>(&b->d_field), need * sizeof(double), b->stream);
      if (e != cudaSuccess) return cuda_fail(e, "tdz_propagate: field buffer");
      b->field_len = need;
    }
    e = cudaMemcpyAsync(b->d_field, field, need * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tdz_propagate: field upload");
    dfield = b->d_field;
  }
  const size_t obs_need = (size_t)b->nruns * nsteps * 5;
  if (b->obs_steps < obs_need) {
    if (b->d_obs) cudaFreeAsync(b->d_obs, b->stream);
    b->d_obs = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void**>(&b->d_obs), obs_need * sizeof(double), b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tdz_propagate: observable buffer");
    b->obs_steps = obs_need;
  }
  if (b->current && b->cur_len < (size_t)b->nruns * nsteps) {
    if (b->d_cur) cudaFreeAsync(b->d_cur, b->stream);
    b->d_cur = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void**>(&b->d_cur), sizeof(double) * b->nruns * nsteps, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tdz_propagate: current buffer");
    b->cur_len = (size_t)b->nruns * nsteps;
  }
  e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tdz_propagate");
  StepArgs a;
  a.geoms = b->d_geoms;
  a.runs = b->d_runs;
  a.lanes = b->d_lanes;
  a.ngroups = b->ngroups;
  a.counter = b->d_counter;
  a.field = dfield;
  a.obs = b->d_obs;
  a.cur = b->current ? b->d_cur : nullptr;
  a.nsteps = nsteps;
  a.step0 = step0;
  a.dt = dt;
  a.tol = b->tol;
  a.max_it = b->max_it;
  e = (b->prec == TDZ_MIXED) ? launch<true>(b, a) : launch<false>(b, a);
  if (e != cudaSuccess) return cuda_fail(e, "tdz_propagate: launch");
  b->last_nsteps = nsteps;
  if (dfield != field) {
    e = cudaStreamSynchronize(b->stream);  // the host field buffer may be reused by the caller
    if (e != cudaSuccess) return cuda_fail(e, "tdz_propagate");
  }
  return TDZ_OK;
}

int tdz_observe(const tdz_batch* b, int run, double* out, int* status) {
  if (!b || run < 0 || run >= b->nruns) return TDZ_EINVAL;
  if (b->nd) return tdz::nd_observe(b->nd, run, out, status, out ? is_device_ptr(out) : false);
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tdz_observe");
  if (out && b->last_nsteps > 0) {
    const size_t cnt = (size_t)b->last_nsteps * 5;
    e = cudaMemcpy(out, b->d_obs + (size_t)run * cnt, cnt * sizeof(double), cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(e, "tdz_observe");
  }
  if (status) {
    int st = 0;
    e = cudaMemcpy(&st, &b->d_runs[run].status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "tdz_observe");
    *status = st;
  }
  return TDZ_OK;
}

int tdz_set_state_all(tdz_batch* b, const double* c) {
  if (!b || !c) return TDZ_EINVAL;
  const bool dev = is_device_ptr(c);
  if (b->nd) {
    long long o = 0;
    for (int r = 0; r < b->nruns; ++r) {
      const int rc = tdz::nd_set_state(b->nd, r, c + 2 * o, dev);
      if (rc != TDZ_OK) return rc;
      o += tdz::nd_run_size(b->nd, r);
    }
    return TDZ_OK;
  }
  const size_t cnt = (size_t)2 * b->total_dof;
  const double* src = c;
  cudaError_t e = cudaSuccess;
  if (!dev) {
    if (!b->d_stage) {
      e = cudaMalloc(&b->d_stage, sizeof(double) * cnt);
      if (e != cudaSuccess) return cuda_fail(e, "tdz_set_state_all: staging buffer");
    }
    e = cudaMemcpyAsync(b->d_stage, c, sizeof(double) * cnt, cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tdz_set_state_all: upload");
    src = b->d_stage;
  }
  cudaMemsetAsync(b->d_bad, 0, sizeof(int), b->stream);
  const int grid = std::min(b->nruns, 148 * 8);
  if (b->prec == TDZ_MIXED)
    k_set_states<true><<<grid, 256, 0, b->stream>>>(src, b->d_off, b->d_runs, b->d_geoms, b->nruns, b->d_bad);
  else
    k_set_states<false><<<grid, 256, 0, b->stream>>>(src, b->d_off, b->d_runs, b->d_geoms, b->nruns, b->d_bad);
  int bad = 0;
  e = cudaMemcpyAsync(&bad, b->d_bad, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tdz_set_state_all");
  if (bad) {
    set_error("tdz_set_state_all: non-finite coefficient");
    return TDZ_ENONFINITE;
  }
  return TDZ_OK;
}

int tdz_observe_all(const tdz_batch* b, double* out, int* status) {
  if (!b) return TDZ_EINVAL;
  if (b->nd) {
    const int cols = 2 + 3 * tdz::nd_dim(b->nd);
    const bool dev = out ? is_device_ptr(out) : false;
    for (int r = 0; r < b->nruns; ++r) {
      const int rc = tdz::nd_observe(b->nd, r, out ? out + (size_t)r * b->last_nsteps * cols : nullptr,
                                     status ? status + r : nullptr, dev);
      if (rc != TDZ_OK) return rc;
    }
    return TDZ_OK;
  }
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tdz_observe_all");
  if (out && b->last_nsteps > 0) {
    e = cudaMemcpy(out, b->d_obs, sizeof(double) * (size_t)b->nruns * b->last_nsteps * 5, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(e, "tdz_observe_all");
  }
  if (status) {
    std::vector<RunDev> r(b->nruns);
    e = cudaMemcpy(r.data(), b->d_runs, sizeof(RunDev) * b->nruns, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "tdz_observe_all");
    for (int k = 0; k < b->nruns; ++k) status[k] = r[k].status;
  }
  return TDZ_OK;
}

int tdz_refine_stats(const tdz_batch* b, double* max_rel_residual, double* mean_solves) {
  if (!b) return TDZ_EINVAL;
  if (b->nd) return tdz::nd_stats(b->nd, max_rel_residual, mean_solves, nullptr);
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tdz_refine_stats");
  std::vector<RunDev> r(b->nruns);
  e = cudaMemcpy(r.data(), b->d_runs, sizeof(RunDev) * b->nruns, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "tdz_refine_stats");
  double mx = 0.0, ns = 0.0;
  for (auto& x : r) {
    mx = std::max(mx, x.max_rel);
    ns += (double)x.nsolve;
  }
  if (max_rel_residual) *max_rel_residual = mx;
  if (mean_solves) *mean_solves = ns;
  return TDZ_OK;
}

int tdz_batch_set_option(tdz_batch* b, int option, int value) {
  if (!b) return TDZ_EINVAL;
  if (option == TDZ_OPT_CURRENT) {
    if (value != 0 && value != 1) return TDZ_EINVAL;
    if (b->nd) {
      set_error("tdz_batch_set_option: the per-step current is recorded by 1-D batches only");
      return TDZ_EUNSUPPORTED;
    }
    if (value == 1 && !b->h_geoms.empty() && !b->h_geoms[0].Mv) {
      // upload the velocity bands in the batch's interleaved layout (binary64, or float2 {hi, lo})
      for (size_t gi = 0; gi < b->h_geoms.size(); ++gi) {
        const auto& G = b->geo[gi];
        const Band& M = b->ops_of[gi]->M;
        const int P1 = b->P + 1;
        const size_t nb = (size_t)G.m * P1 * G.ks;
        std::vector<double> hv(nb, 0.0);
        for (int k = 0; k < G.K; ++k)
          for (int i = 0; i < G.m; ++i) {
            const int64_t gr = (int64_t)k * G.m + i;
            if (gr >= G.n) continue;
            for (int d = 1; d <= b->P && gr - d >= 0; ++d) hv[((size_t)i * P1 + d) * G.ks + k] = M.at(gr, d);
          }
        void* dst = nullptr;
        if (b->prec == TDZ_MIXED) {
          std::vector<float> hf(2 * nb);
          for (size_t q = 0; q < nb; ++q) {
            hf[2 * q] = (float)hv[q];
            hf[2 * q + 1] = (float)(hv[q] - (double)(float)hv[q]);
          }
          dst = b->alloc(nb * 8);
          if (dst && cudaMemcpyAsync(dst, hf.data(), nb * 8, cudaMemcpyHostToDevice, b->stream) != cudaSuccess) dst = nullptr;
          if (dst && cudaStreamSynchronize(b->stream) != cudaSuccess) dst = nullptr;
        } else {
          dst = b->alloc(nb * 8);
          if (dst && cudaMemcpyAsync(dst, hv.data(), nb * 8, cudaMemcpyHostToDevice, b->stream) != cudaSuccess) dst = nullptr;
          if (dst && cudaStreamSynchronize(b->stream) != cudaSuccess) dst = nullptr;
        }
        if (!dst) {
          set_error("tdz_batch_set_option: velocity band upload failed");
          return TDZ_ENOMEM;
        }
        b->h_geoms[gi].Mv = dst;
      }
      cudaError_t e = cudaMemcpyAsync(b->d_geoms, b->h_geoms.data(), sizeof(GeomDev) * b->h_geoms.size(),
                                      cudaMemcpyHostToDevice, b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
      if (e != cudaSuccess) return cuda_fail(e, "tdz_batch_set_option");
    }
    b->current = value == 1;
    return TDZ_OK;
  }
  if (b->nd) return tdz::nd_set_option(b->nd, option, value);
  if (option == TDZ_OPT_PRECOND && value >= TDZ_PRECOND_AUTO && value <= TDZ_PRECOND_FD) return TDZ_OK;
  if (option == TDZ_OPT_OPERATOR && value >= TDZ_OPERATOR_AUTO && value <= TDZ_OPERATOR_STENCIL) return TDZ_OK;
  if (option == TDZ_OPT_APPLY_GROUPS && (value == 0 || value == 8 || value == 16)) return TDZ_OK;
  if (option == TDZ_OPT_WAIT_TEST && (value == 0 || value == 1)) return TDZ_OK;
  return TDZ_EINVAL;
}

int tdz_observe_current(const tdz_batch* b, int run, double* out) {
  if (!b || !out || run < 0 || run >= b->nruns) return TDZ_EINVAL;
  if (b->nd || !b->current || !b->d_cur || b->last_nsteps < 1) {
    set_error("tdz_observe_current: no current recorded (1-D batch with TDZ_OPT_CURRENT set before tdz_propagate)");
    return TDZ_EINVAL;
  }
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(out, b->d_cur + (size_t)run * b->last_nsteps, sizeof(double) * b->last_nsteps, cudaMemcpyDefault);
  if (e != cudaSuccess) return cuda_fail(e, "tdz_observe_current");
  return TDZ_OK;
}

int tdz_batch_tuning(const tdz_batch* b, int geometry, int* groups, double* ms) {
  if (!b || geometry < 0) return TDZ_EINVAL;
  if (b->nd) return tdz::nd_tuning(b->nd, geometry, groups, ms);
  if (groups) *groups = 0;
  if (ms) ms[0] = ms[1] = 0.0;
  return TDZ_OK;
}

int tdz_batch_precond_tuning(const tdz_batch* b, int geometry, int* variant, double* ms) {
  if (!b || geometry < 0) return TDZ_EINVAL;
  if (b->nd) return tdz::nd_precond_tuning(b->nd, geometry, variant, ms);
  if (variant) *variant = -1;
  if (ms)
    for (int c = 0; c < 4; ++c) ms[c] = 0.0;
  return TDZ_OK;
}

int tdz_batch_time_operator(tdz_batch* b, int geometry, int reps, double* ms) {
  if (!b || !ms || geometry < 0 || reps < 1) return TDZ_EINVAL;
  if (!b->nd) return TDZ_EUNSUPPORTED;
  return tdz::nd_time_operator(b->nd, geometry, reps, ms);
}

int tdz_batch_ground_state(tdz_batch* b, int run, double sigma, double tol, int max_outer, double* energy,
                           int* iterations, double* residual) {
  if (!b) return TDZ_EINVAL;
  if (!b->nd) return TDZ_EUNSUPPORTED;
  return tdz::nd_ground_state(b->nd, run, sigma, tol, max_outer, energy, iterations, residual);
}

int tdz_krylov_stats(const tdz_batch* b, double* iterations) {
  if (!b || !iterations) return TDZ_EINVAL;
  *iterations = 0.0;
  if (b->nd) return tdz::nd_stats(b->nd, nullptr, nullptr, iterations);
  return TDZ_OK;
}

void tdz_batch_destroy(tdz_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  delete b;
}

}  // extern "C"

// ============================================================================ allocation-free variant
// Scratch for tdz_cn1d_propagate_noalloc: one binary64 run of at most TDZ_NOALLOC_MAX_N coefficients
// and degree <= 8, in a fixed device array that every GPU loading this library holds until exit.
namespace tdz {
constexpr int NOALLOC_ROWS = TDZ_NOALLOC_MAX_N + 32;                       // interleaved rows m*32 bound
constexpr size_t NOALLOC_DOUBLES = (size_t)NOALLOC_ROWS * (7 * MAXP + 15) + 64;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

struct NoAllocLayout {
  int n, m, K, P;
  size_t band, state, rhs, Lc, Dv, gd, dl, desc;  // offsets in doubles
};

// Pack the caller's natural-order bands and state into the interleaved [row][lane] layout and
// write the run descriptors; everything the step kernel reads before writing is set here.
__global__ void noalloc_pack(double* scr, NoAllocLayout L, const double* bands, const double* state) {
  const int P1 = L.P + 1;
  const size_t rows = (size_t)L.m * LANES;
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = tid; e < 5 * rows * P1; e += stride) {
    const int q = (int)(e / (rows * P1));
    const size_t rem = e % (rows * P1);
    const int i = (int)(rem / ((size_t)P1 * LANES));
    const int d = (int)((rem / LANES) % P1);
    const int k = (int)(rem % LANES);
    const long long g = (long long)k * L.m + i;
    double v = 0.0;
    if (k < L.K) {
      if (g < L.n) {
        if (g - d >= 0) v = bands[((size_t)q * L.n + g) * P1 + d];
      } else if (q == 0 && d == 0) {
        v = 1.0;  // padding rows: identity in S
      }
    }
    scr[L.band + e] = v;
  }
  for (size_t e = tid; e < rows; e += stride) {
    const int i = (int)(e / LANES), k = (int)(e % LANES);
    const long long g = (long long)k * L.m + i;
    const bool in = k < L.K && g < L.n;
    scr[L.state + 2 * e] = in ? state[2 * g] : 0.0;
    scr[L.state + 2 * e + 1] = in ? state[2 * g + 1] : 0.0;
  }
  if (tid == 0) {
    GeomDev* G = reinterpret_cast<GeomDev*>(scr + L.desc);
    RunDev* R = reinterpret_cast<RunDev*>(G + 1);
    int* lanes = reinterpret_cast<int*>(R + 1);
    const size_t nb = rows * P1;
    *G = GeomDev{L.n, L.m, L.K, LANES, scr + L.band, scr + L.band + nb, scr + L.band + 2 * nb, scr + L.band + 3 * nb,
                 scr + L.band + 4 * nb, nullptr, nullptr};
    RunDev r{};
    r.geom = 0;
    r.status = TDZ_OK;
    r.state = scr + L.state;
    r.rhs = scr + L.rhs;
    r.Lc = scr + L.Lc;
    r.Dv = scr + L.Dv;
    r.gd = scr + L.gd;
    r.dl = scr + L.dl;
    *R = r;
    for (int k = 0; k < LANES; ++k) lanes[k] = k < L.K ? k : -1;  // run 0, lane k (one warp)
    lanes[LANES] = 0;                                             // work counter
  }
}

__global__ void noalloc_unpack(const double* scr, NoAllocLayout L, double* state) {
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (size_t g = tid; g < (size_t)L.n; g += (size_t)gridDim.x * blockDim.x) {
    const size_t e = (size_t)(g % L.m) * LANES + g / L.m;
    state[2 * g] = scr[L.state + 2 * e];
    state[2 * g + 1] = scr[L.state + 2 * e + 1];
  }
}

static double* g_noalloc_ptr[64] = {nullptr};
static std::mutex g_noalloc_mu;

template <int P>
cudaError_t noalloc_launch(cudaStream_t st, const StepArgs& a) {
  const size_t sm = block_smem(P, false, LANES);
  cudaError_t e = ensure_smem<P, false, false>(sm);
  if (e != cudaSuccess) return e;
  cn1d_kernel<P, false, false><<<1, LANES, sm, st>>>(a);
  return cudaGetLastError();
}
}  // namespace tdz

extern "C" int tdz_cn1d_propagate_noalloc(const double* bands, int64_t n, int degree, const double* field, double dt,
                                          int64_t step0, int64_t nsteps, double* state, double* obs, void* cuda_stream,
                                          int* status) {
  using namespace tdz;
  if (!bands || !field || !state || !obs || degree < 1 || degree > MAXP || n < degree + 1 || nsteps < 1 ||
      step0 < 0 || !(dt > 0) || !std::isfinite(dt)) {
    set_error("tdz_cn1d_propagate_noalloc: bad arguments");
    return TDZ_EINVAL;
  }
  if (n > TDZ_NOALLOC_MAX_N) {
    set_error("tdz_cn1d_propagate_noalloc: n exceeds TDZ_NOALLOC_MAX_N (" + std::to_string(TDZ_NOALLOC_MAX_N) +
              "); use the batch API for larger runs");
    return TDZ_EINVAL;
  }
  const int P = degree;
  NoAllocLayout L{};
  L.n = (int)n;
  L.P = P;
  L.K = std::max(1, std::min(32, (int)n / (3 * P)));
  L.m = (int)((n + L.K - 1) / L.K);
  while (L.K > 1 && L.m - P < P + 1) {
    --L.K;
    L.m = (int)((n + L.K - 1) / L.K);
  }
  const size_t rows = (size_t)L.m * LANES;
  if (rows > (size_t)NOALLOC_ROWS) {
    set_error("tdz_cn1d_propagate_noalloc: the interleaved layout of this size exceeds the static scratch");
    return TDZ_EINVAL;
  }
  L.band = 0;
  L.state = L.band + 5 * rows * (P + 1);
  L.rhs = L.state + 2 * rows;
  L.Lc = L.rhs + 2 * rows;
  L.Dv = L.Lc + 2 * rows * P;
  L.gd = L.Dv + 2 * rows;
  L.dl = L.gd + 2 * rows;
  L.desc = L.dl + 2 * rows;
  L.desc = (L.desc + 31) & ~(size_t)31;
  if (L.desc + 64 > NOALLOC_DOUBLES) {
    set_error("tdz_cn1d_propagate_noalloc: scratch layout overflow");
    return TDZ_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "tdz_cn1d_propagate_noalloc: device");
  if (dev < 0 || dev >= 64) {
    set_error("tdz_cn1d_propagate_noalloc: device index " + std::to_string(dev) + " beyond the 64 devices supported");
    return TDZ_EINVAL;
  }
  double* scr = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // first call on this device (which is current): resolve the device address of the array
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "tdz_cn1d_propagate_noalloc: cudaGetSymbolAddress");
      g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    scr = g_noalloc_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  noalloc_pack<<<148, 256, 0, st>>>(scr, L, bands, state);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tdz_cn1d_propagate_noalloc: pack");
  GeomDev* G = reinterpret_cast<GeomDev*>(scr + L.desc);
  RunDev* R = reinterpret_cast<RunDev*>(G + 1);
  int* lanes = reinterpret_cast<int*>(R + 1);
  StepArgs a;
  a.geoms = G;
  a.runs = R;
  a.lanes = lanes;
  a.ngroups = 1;
  a.counter = lanes + LANES;
  a.field = field;
  a.obs = obs;
  a.cur = nullptr;
  a.nsteps = nsteps;
  a.step0 = step0;
  a.dt = dt;
  a.tol = 1e-11;
  a.max_it = 1;
  switch (P) {
    case 1: e = noalloc_launch<1>(st, a); break;
    case 2: e = noalloc_launch<2>(st, a); break;
    case 3: e = noalloc_launch<3>(st, a); break;
    case 4: e = noalloc_launch<4>(st, a); break;
    case 5: e = noalloc_launch<5>(st, a); break;
    case 6: e = noalloc_launch<6>(st, a); break;
    case 7: e = noalloc_launch<7>(st, a); break;
    default: e = noalloc_launch<8>(st, a); break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "tdz_cn1d_propagate_noalloc: propagate");
  noalloc_unpack<<<64, 256, 0, st>>>(scr, L, state);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tdz_cn1d_propagate_noalloc: unpack");
  if (status) {
    int sv = 0;
    e = cudaMemcpyAsync(&sv, &R->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "tdz_cn1d_propagate_noalloc: status");
    *status = sv;
  }
  return TDZ_OK;
}
