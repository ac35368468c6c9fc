// Internal declarations shared by the host (C++) and device (CUDA) translation units.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "tdz.h"

namespace tdz {

void set_error(const std::string& msg);
// autotuner cache in the file named by TDZ_TUNE_CACHE (absent: no cache)
bool tune_cache_get(const std::string& key, std::vector<double>& values);
void tune_cache_put(const std::string& key, const std::vector<double>& values);

struct Basis {
  std::vector<double> knots;
  int p = 0;        // degree
  int nq = 0;       // Gauss points per element
  int64_t nfun = 0; // B-splines incl. Dirichlet ends
  // per element e: span index, quadrature points, weights (w*J), values and derivatives
  std::vector<int64_t> span;           // nelem
  std::vector<double> xq, wq;          // nelem*nq
  std::vector<double> val, der;        // nelem*nq*(p+1), column r <-> function span-p+r
  int64_t nelem() const { return (int64_t)span.size(); }
};

struct Medium {
  int mass_kind = TDZ_MASS_CONST, pot_kind = TDZ_POT_ZERO;
  double mass_par[4] = {1, 0, 0, 0};
  double pot_par[4] = {0, 0, 0, 0};
  std::vector<double> bounds, lmass, lpot;
  int cap_kind = TDZ_CAP_NONE;
  double cap_par[4] = {0, 0, 0, 0};
  double inv_mass(const double* r, int dim) const;
  double potential(const double* r, int dim) const;
  double dpotential(const double* r, int dim, int axis) const;
  double cap_axis(double x) const;  // 1-D absorbing mask of one coordinate (eta = sum over the axes)
};

// symmetric lower band: band[i*(p+1)+d] = M(i, i-d)
struct Band {
  int64_t n = 0;
  int p = 0;
  std::vector<double> a;
  double at(int64_t i, int d) const { return a[(size_t)i * (p + 1) + d]; }
};

struct Ops {
  int dim = 1;
  int64_t n[3] = {0, 0, 0};
  int p[3] = {0, 0, 0};
  Medium med;
  // 1-D matrices (W: absorbing-layer mask, all zero without one; M: the real antisymmetric part of the
  // velocity matrix, Vel = -(i/2) M, stored as its lower band M(i, i-d), d >= 1)
  Band S, T, V, H0, D, G, K, W, M;
  // 2-D / 3-D: per-axis 1-D factors (unit-mass kinetic T1 = 1/2 <N'|N'>, the axis' absorbing mask W_a)
  // and quadrature tables
  Band Sa[3], T1a[3], Da[3], Wa[3];
  bool has_cap() const { return med.cap_kind != TDZ_CAP_NONE; }
  Basis axis[3];
};

// 2-D / 3-D batches (tdz_nd.cu), reached through the public tdz_batch_* entry points
struct NdBatch;
int nd_batch_create(const tdz_ops* const* ops, int nops, int nruns, const int* ops_index, int precision, void* stream,
                    NdBatch** out);
void nd_batch_destroy(NdBatch* b);
long long nd_run_size(const NdBatch* b, int run);
int nd_set_state(NdBatch* b, int run, const double* c, bool device);
int nd_get_state(const NdBatch* b, int run, double* c, bool device);
int nd_propagate(NdBatch* b, const double* field_host, double dt, long long step0, long long nsteps);
int nd_observe(const NdBatch* b, int run, double* out, int* status, bool device);
int nd_stats(const NdBatch* b, double* max_rel, double* solves, double* iters);
void nd_set_refinement(NdBatch* b, double tol, int max_it);
int nd_set_option(NdBatch* b, int option, int value);
int nd_tuning(const NdBatch* b, int geometry, int* groups, double* ms);
int nd_precond_tuning(const NdBatch* b, int geometry, int* variant, double* ms);
int nd_time_operator(NdBatch* b, int geometry, int reps, double* ms);
int nd_ground_state(NdBatch* b, int run, double sigma, double tol, int max_outer, double* energy, int* outer,
                    double* resid);
int nd_dim(const NdBatch* b);
size_t nd_device_bytes(const NdBatch* b);

// One axis transform of the mixed-precision fast-diagonalisation preconditioner on the tensor cores
// (tdz_tc.cu; semantics of tdz_tc_axis_transform, asynchronous on `st`, a run-out wait sets *err)
int tc_axis_transform(const float* a_hi, const float* a_lo, long long rows, int K, const float* b, const float* b_lo,
                      int ncols, long long plane_rows, long long plane_stride, float* out_hi, float* out_lo, int* err,
                      int tile_n, struct CUstream_st* st);

}  // namespace tdz

struct tdz_basis { tdz::Basis b; };
struct tdz_ops { tdz::Ops o; };
