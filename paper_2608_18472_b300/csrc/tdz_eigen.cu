// Lowest eigenpairs of the 1-D generalised eigenproblem H0 c = eps S c (Eq. gen_ev) for a batch of
// geometries on the GPU, by subspace inverse iteration with Rayleigh-Ritz (binary64 throughout).
//
// Per geometry (one warp each):
//   * a shift sigma below the spectrum (a little under min_i V_ii / S_ii), so F = H0 - sigma S is
//     positive definite and its band LDL^T needs no pivoting; F is factored once;
//   * a block X of k = nstates + 2 vectors (the two guard vectors carry the convergence of the wanted
//     ones past near-degenerate pairs, e.g. the tunnelling doublet of a double well);
//   * every iteration: Y = F^-1 S X, then Rayleigh-Ritz in span(Y): the k x k pencil (Y^T H0 Y,
//     Y^T S Y) is reduced by a Cholesky factor of Y^T S Y and diagonalised by cyclic Jacobi rotations;
//     X <- Y U (the Ritz vectors, S-orthonormal), until the wanted Ritz pairs' residuals
//     ||H0 x - eps S x|| / ||eps S x|| are below 1e-11;
//   * phase convention of Sec. "Wavefunction realignment": real, S-normalised, largest component
//     positive.
// The band arrays are the natural-order lower bands M(i, i-d) of tdz_ops_band.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tdz_internal.h"

namespace tdz {
namespace {

constexpr int KMAX = 8;

struct EigGeom {
  int n;
  double sigma;
  const double* S;   // [n][P+1]
  const double* H;   // [n][P+1]
  double* F;         // [n][P+1] factor of H - sigma S (L below the diagonal, D on it)
  double* X;         // [k][n]
  double* Y;         // [k][n]
  double* Z;         // [k][n] scratch (S X, then H Y / S Y)
  double* theta;     // [k] Ritz values
  double* resid;     // [k] relative residuals
  int* iters;
  int* status;
};

template <int P>
__device__ double band_row(const double* M, int n, int i, const double* x) {
  // (M x)_i for a symmetric band stored as the lower band
  double s = M[(size_t)i * (P + 1)] * x[i];
#pragma unroll
  for (int d = 1; d <= P; ++d) {
    if (i - d >= 0) s = fma(M[(size_t)i * (P + 1) + d], x[i - d], s);
    if (i + d < n) s = fma(M[(size_t)(i + d) * (P + 1) + d], x[i + d], s);
  }
  return s;
}

__device__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// cyclic Jacobi diagonalisation of the symmetric k x k matrix C (in place: its diagonal -> eigenvalues),
// V <- eigenvectors (columns); single thread
__device__ void jacobi(double (*C)[KMAX], double (*V)[KMAX], int k) {
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) V[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < k; ++i) {
      diag += C[i][i] * C[i][i];
      for (int j = i + 1; j < k; ++j) off += C[i][j] * C[i][j];
    }
    if (off <= 1e-32 * diag) break;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = C[p][q];
        if (fabs(apq) < 1e-300) continue;
        const double tt = (C[q][q] - C[p][p]) / (2.0 * apq);
        const double t = (tt >= 0 ? 1.0 : -1.0) / (fabs(tt) + sqrt(1.0 + tt * tt));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int r = 0; r < k; ++r) {  // columns p, q
          const double crp = C[r][p], crq = C[r][q];
          C[r][p] = c * crp - s * crq;
          C[r][q] = s * crp + c * crq;
        }
        for (int r = 0; r < k; ++r) {  // rows p, q
          const double cpr = C[p][r], cqr = C[q][r];
          C[p][r] = c * cpr - s * cqr;
          C[q][r] = s * cpr + c * cqr;
        }
        for (int r = 0; r < k; ++r) {
          const double vrp = V[r][p], vrq = V[r][q];
          V[r][p] = c * vrp - s * vrq;
          V[r][q] = s * vrp + c * vrq;
        }
      }
  }
}

template <int P>
__global__ void k_lowest_states(EigGeom* geoms, int ngeom, int k, int nwanted, int maxit) {
  const int g = blockIdx.x;
  if (g >= ngeom) return;
  const int lane = threadIdx.x;
  EigGeom G = geoms[g];
  const int n = G.n;
  __shared__ double sA[KMAX][KMAX], sB[KMAX][KMAX], sU[KMAX][KMAX], sth[KMAX];
  __shared__ double sl[P + 1];
  __shared__ int s_ok;
  // ---- factor F = H - sigma S in place: right-looking band LDL^T (positive definite, no pivoting)
  for (size_t e = lane; e < (size_t)n * (P + 1); e += 32) G.F[e] = G.H[e] - G.sigma * G.S[e];
  __syncwarp();
  for (int j = 0; j < n; ++j) {
    const double dj = G.F[(size_t)j * (P + 1)];
    const int rmax = min(P, n - 1 - j);
    if (lane >= 1 && lane <= rmax) sl[lane] = G.F[(size_t)(j + lane) * (P + 1) + lane] / dj;
    __syncwarp();
    // entries (j + r, j + c), 1 <= c <= r <= rmax, one per lane
    for (int t = lane; t < P * (P + 1) / 2; t += 32) {
      int r = 1, c = t;
      while (c >= r) {
        c -= r;
        ++r;
      }
      c += 1;  // 1 <= c <= r
      if (r <= rmax) G.F[(size_t)(j + r) * (P + 1) + (r - c)] -= sl[r] * sl[c] * dj;
    }
    __syncwarp();
    if (lane >= 1 && lane <= rmax) G.F[(size_t)(j + lane) * (P + 1) + lane] = sl[lane];
    __syncwarp();
  }
  // ---- starting block: smooth sine modes
  for (int v = 0; v < k; ++v)
    for (int i = lane; i < n; i += 32) G.X[(size_t)v * n + i] = sin(M_PI * (double)(v + 1) * (double)(i + 1) / (double)(n + 1));
  __syncwarp();
  if (lane == 0) s_ok = 0;
  __syncwarp();
  int it = 0;
  for (; it < maxit; ++it) {
    // Z = S X
    for (int v = 0; v < k; ++v)
      for (int i = lane; i < n; i += 32) G.Z[(size_t)v * n + i] = band_row<P>(G.S, n, i, G.X + (size_t)v * n);
    __syncwarp();
    // Y = F^-1 Z: lanes 0..k-1 each solve one column (L y = z, y /= D, L^T y = y)
    if (lane < k) {
      double* y = G.Y + (size_t)lane * n;
      const double* z = G.Z + (size_t)lane * n;
      for (int i = 0; i < n; ++i) {
        double s = z[i];
#pragma unroll
        for (int d = 1; d <= P; ++d)
          if (i - d >= 0) s -= G.F[(size_t)i * (P + 1) + d] * y[i - d];
        y[i] = s;
      }
      for (int i = 0; i < n; ++i) y[i] /= G.F[(size_t)i * (P + 1)];
      for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
#pragma unroll
        for (int d = 1; d <= P; ++d)
          if (i + d < n) s -= G.F[(size_t)(i + d) * (P + 1) + d] * y[i + d];
        y[i] = s;
      }
    }
    __syncwarp();
    // Rayleigh-Ritz: A = Y^T H Y, B = Y^T S Y
    for (int a = 0; a < k; ++a) {
      for (int i = lane; i < n; i += 32) G.Z[(size_t)a * n + i] = band_row<P>(G.H, n, i, G.Y + (size_t)a * n);
    }
    __syncwarp();
    for (int a = 0; a < k; ++a)
      for (int c = 0; c <= a; ++c) {
        double sa = 0.0;
        for (int i = lane; i < n; i += 32) sa += G.Y[(size_t)c * n + i] * G.Z[(size_t)a * n + i];
        sa = warp_sum(sa);
        if (lane == 0) sA[a][c] = sA[c][a] = sa;
      }
    __syncwarp();
    for (int a = 0; a < k; ++a)
      for (int i = lane; i < n; i += 32) G.Z[(size_t)a * n + i] = band_row<P>(G.S, n, i, G.Y + (size_t)a * n);
    __syncwarp();
    for (int a = 0; a < k; ++a)
      for (int c = 0; c <= a; ++c) {
        double sb = 0.0;
        for (int i = lane; i < n; i += 32) sb += G.Y[(size_t)c * n + i] * G.Z[(size_t)a * n + i];
        sb = warp_sum(sb);
        if (lane == 0) sB[a][c] = sB[c][a] = sb;
      }
    __syncwarp();
    if (lane == 0) {
      // B = R R^T (Cholesky, lower R); C = R^-1 A R^-T; C = V diag V^T; U = R^-T V
      double R[KMAX][KMAX] = {};
      bool ok = true;
      for (int i = 0; i < k && ok; ++i)
        for (int j = 0; j <= i; ++j) {
          double s = sB[i][j];
          for (int q = 0; q < j; ++q) s -= R[i][q] * R[j][q];
          if (i == j) {
            if (!(s > 0.0)) ok = false;
            else R[i][i] = sqrt(s);
          } else {
            R[i][j] = s / R[j][j];
          }
        }
      if (!ok) {
        s_ok = -1;
      } else {
        double Tm[KMAX][KMAX], Cm[KMAX][KMAX], V[KMAX][KMAX];
        for (int j = 0; j < k; ++j)  // Tm = R^-1 A (columns of A)
          for (int i = 0; i < k; ++i) {
            double s = sA[i][j];
            for (int q = 0; q < i; ++q) s -= R[i][q] * Tm[q][j];
            Tm[i][j] = s / R[i][i];
          }
        for (int i = 0; i < k; ++i)  // Cm = Tm R^-T  (solve Cm R^T = Tm row-wise)
          for (int j = 0; j < k; ++j) {
            double s = Tm[i][j];
            for (int q = 0; q < j; ++q) s -= Cm[i][q] * R[j][q];
            Cm[i][j] = s / R[j][j];
          }
        for (int i = 0; i < k; ++i)
          for (int j = 0; j < i; ++j) Cm[i][j] = Cm[j][i] = 0.5 * (Cm[i][j] + Cm[j][i]);
        jacobi(Cm, V, k);
        // sort ascending
        int ord[KMAX];
        for (int i = 0; i < k; ++i) ord[i] = i;
        for (int i = 1; i < k; ++i)
          for (int j = i; j > 0 && Cm[ord[j]][ord[j]] < Cm[ord[j - 1]][ord[j - 1]]; --j) {
            const int t = ord[j];
            ord[j] = ord[j - 1];
            ord[j - 1] = t;
          }
        for (int c = 0; c < k; ++c) {
          sth[c] = Cm[ord[c]][ord[c]];
          for (int i = k - 1; i >= 0; --i) {  // U[:, c] = R^-T V[:, ord[c]]
            double s = V[i][ord[c]];
            for (int q = i + 1; q < k; ++q) s -= R[q][i] * sU[q][c];
            sU[i][c] = s / R[i][i];
          }
        }
        s_ok = 0;
      }
    }
    __syncwarp();
    if (s_ok < 0) break;
    // X = Y U
    for (int i = lane; i < n; i += 32) {
      double yv[KMAX];
      for (int a = 0; a < k; ++a) yv[a] = G.Y[(size_t)a * n + i];
      for (int c = 0; c < k; ++c) {
        double s = 0.0;
        for (int a = 0; a < k; ++a) s = fma(yv[a], sU[a][c], s);
        G.X[(size_t)c * n + i] = s;
      }
    }
    __syncwarp();
    // converged when every wanted Ritz pair has ||H x - eps S x|| <= 1e-11 ||eps S x||
    double worst = 0.0;
    for (int c = 0; c < nwanted; ++c) {
      const double* x = G.X + (size_t)c * n;
      double rr = 0.0, bb = 0.0;
      for (int i = lane; i < n; i += 32) {
        const double sx = band_row<P>(G.S, n, i, x), hx = band_row<P>(G.H, n, i, x);
        const double r = hx - sth[c] * sx;
        rr += r * r;
        bb += sth[c] * sth[c] * sx * sx;
      }
      rr = warp_sum(rr);
      bb = warp_sum(bb);
      worst = fmax(worst, sqrt(rr / fmax(bb, 1e-300)));
    }
    if (worst <= 1e-11) {
      if (lane == 0) s_ok = 1;
      __syncwarp();
      break;
    }
  }
  // residuals ||H x - eps S x|| / ||eps S x|| of the wanted Ritz pairs, normalisation and sign
  for (int c = 0; c < nwanted; ++c) {
    const double* x = G.X + (size_t)c * n;
    double rr = 0.0, bb = 0.0, nn = 0.0, big = 0.0;
    int ibig = 0;
    for (int i = lane; i < n; i += 32) {
      const double sx = band_row<P>(G.S, n, i, x), hx = band_row<P>(G.H, n, i, x);
      const double r = hx - sth[c] * sx;
      rr += r * r;
      bb += sth[c] * sth[c] * sx * sx;
      nn += x[i] * sx;
      if (fabs(x[i]) > big) {
        big = fabs(x[i]);
        ibig = i;
      }
    }
    rr = warp_sum(rr);
    bb = warp_sum(bb);
    nn = warp_sum(nn);
    for (int o = 16; o > 0; o >>= 1) {  // index of the largest component (first on ties)
      const double ob = __shfl_xor_sync(0xffffffffu, big, o);
      const int oi = __shfl_xor_sync(0xffffffffu, ibig, o);
      if (ob > big || (ob == big && oi < ibig)) {
        big = ob;
        ibig = oi;
      }
    }
    const double scale = (x[ibig] < 0 ? -1.0 : 1.0) / sqrt(nn);
    __syncwarp();
    for (int i = lane; i < n; i += 32) G.X[(size_t)c * n + i] *= scale;
    if (lane == 0) {
      G.theta[c] = sth[c];
      G.resid[c] = sqrt(rr / fmax(bb, 1e-300));
    }
    __syncwarp();
  }
  if (lane == 0) {
    *G.iters = it + 1;
    *G.status = s_ok == 1 ? TDZ_OK : TDZ_ENOCONV;
  }
}

int fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return TDZ_ECUDA;
}

template <int P>
void launch(EigGeom* d, int ng, int k, int nw, int maxit, cudaStream_t st) {
  k_lowest_states<P><<<ng, 32, 0, st>>>(d, ng, k, nw, maxit);
}

}  // namespace
}  // namespace tdz

using namespace tdz;

extern "C" int tdz_lowest_states(const tdz_ops* const* ops, int nops, int nstates, double* energies, double* states,
                                 double* residuals, int* iterations, void* cuda_stream) {
  if (!ops || nops < 1 || nstates < 1 || nstates > KMAX - 2 || !energies || !states) {
    set_error("tdz_lowest_states: bad arguments (1 <= nstates <= 6)");
    return TDZ_EINVAL;
  }
  const int P = ops[0] ? ops[0]->o.p[0] : 0;
  for (int g = 0; g < nops; ++g) {
    if (!ops[g] || ops[g]->o.dim != 1 || ops[g]->o.p[0] != P || ops[g]->o.n[0] < nstates + 2) {
      set_error("tdz_lowest_states: 1-D operators of one degree with at least nstates + 2 coefficients");
      return TDZ_EINVAL;
    }
  }
  if (P < 1 || P > 8) return TDZ_EUNSUPPORTED;
  const int k = nstates + 2;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // device storage: per geometry S, H (uploaded), F, X, Y, Z, theta, resid, iters, status
  std::vector<EigGeom> hg(nops);
  size_t total = 0;
  std::vector<size_t> off(nops);
  for (int g = 0; g < nops; ++g) {
    const size_t n = (size_t)ops[g]->o.n[0];
    off[g] = total;
    total += 3 * n * (P + 1) + 3 * (size_t)k * n + 2 * (size_t)k + 2;
  }
  double* dbuf = nullptr;
  EigGeom* dgeo = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&dbuf), sizeof(double) * total, st);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&dgeo), sizeof(EigGeom) * nops, st);
  if (e != cudaSuccess) {
    if (dbuf) cudaFreeAsync(dbuf, st);
    return fail(e, "tdz_lowest_states: device memory");
  }
  std::vector<double> hostbuf(total, 0.0);
  for (int g = 0; g < nops; ++g) {
    const Ops& o = ops[g]->o;
    const size_t n = (size_t)o.n[0], nb = n * (P + 1);
    double* base = hostbuf.data() + off[g];
    std::copy(o.S.a.begin(), o.S.a.end(), base);
    std::copy(o.H0.a.begin(), o.H0.a.end(), base + nb);
    // shift below the spectrum: E0 >= min over the domain of V > min_i V_ii / S_ii - spread (Galerkin
    // levels are bounded below by the potential's minimum); a margin of 1e-3 of the diagonal spread
    double vmin = 1e300, vmax = -1e300;
    for (size_t i = 0; i < n; ++i) {
      const double v = o.V.at((int64_t)i, 0) / o.S.at((int64_t)i, 0);
      vmin = std::min(vmin, v);
      vmax = std::max(vmax, v);
    }
    double* d = dbuf + off[g];
    hg[g] = EigGeom{(int)n, vmin - 1e-3 * (vmax - vmin) - 1e-9 * (1.0 + std::fabs(vmin)), d, d + nb, d + 2 * nb,
                    d + 3 * nb, d + 3 * nb + k * n, d + 3 * nb + 2 * k * n, d + 3 * nb + 3 * k * n,
                    d + 3 * nb + 3 * k * n + k, reinterpret_cast<int*>(d + 3 * nb + 3 * k * n + 2 * k),
                    reinterpret_cast<int*>(d + 3 * nb + 3 * k * n + 2 * k + 1)};
  }
  e = cudaMemcpyAsync(dbuf, hostbuf.data(), sizeof(double) * total, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dgeo, hg.data(), sizeof(EigGeom) * nops, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    switch (P) {
      case 1: launch<1>(dgeo, nops, k, nstates, 2000, st); break;
      case 2: launch<2>(dgeo, nops, k, nstates, 2000, st); break;
      case 3: launch<3>(dgeo, nops, k, nstates, 2000, st); break;
      case 4: launch<4>(dgeo, nops, k, nstates, 2000, st); break;
      case 5: launch<5>(dgeo, nops, k, nstates, 2000, st); break;
      case 6: launch<6>(dgeo, nops, k, nstates, 2000, st); break;
      case 7: launch<7>(dgeo, nops, k, nstates, 2000, st); break;
      default: launch<8>(dgeo, nops, k, nstates, 2000, st); break;
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hostbuf.data(), dbuf, sizeof(double) * total, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(dbuf, st);
  cudaFreeAsync(dgeo, st);
  cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e, "tdz_lowest_states");
  int rc = TDZ_OK;
  size_t so = 0;
  for (int g = 0; g < nops; ++g) {
    const size_t n = (size_t)ops[g]->o.n[0], nb = n * (P + 1);
    const double* base = hostbuf.data() + off[g];
    const double* X = base + 3 * nb;
    const double* theta = base + 3 * nb + 3 * k * n;
    const double* resid = theta + k;
    int it = 0, stat = 0;
    std::memcpy(&it, base + 3 * nb + 3 * k * n + 2 * k, sizeof(int));
    std::memcpy(&stat, base + 3 * nb + 3 * k * n + 2 * k + 1, sizeof(int));
    for (int c = 0; c < nstates; ++c) {
      energies[(size_t)g * nstates + c] = theta[c];
      if (residuals) residuals[(size_t)g * nstates + c] = resid[c];
      for (size_t i = 0; i < n; ++i) {
        states[so + 2 * i] = X[(size_t)c * n + i];
        states[so + 2 * i + 1] = 0.0;
      }
      so += 2 * n;
    }
    if (iterations) iterations[g] = it;
    if (stat != TDZ_OK) rc = TDZ_ENOCONV;
  }
  if (rc != TDZ_OK) set_error("tdz_lowest_states: some geometry did not converge within the iteration cap");
  return rc;
}
