// Host side of the TDSE-Z B300 library: Gauss-Legendre rules, B-spline tables,
// medium evaluation, one-pass Galerkin band assembly and the 1-D ground state.
//
// Paper references (arXiv 2608.18472):
//   Sec. "Weak form"          open knot vectors, Dirichlet by dropping the end functions, Eq. tensor3d
//   Sec. "Parallel assembly"  Gauss quadrature per knot span, Eqs. mass_elem, bdd_elem, potential and
//                             dipole element formulas; all matrices in one fused pass
//   Sec. "Dipoles"            Eq. pdm_acceleration (G = <m^-1 dV>, K = <m^-1> matrices)
//   Eq. gen_ev                ground state for the initial condition
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "tdz_internal.h"

namespace tdz {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

// ----------------------------------------------------------------------------- autotuner cache
// One JSON object per line, {"key": "...", "values": [v0, v1, ...]}, in the file named by the
// environment variable TDZ_TUNE_CACHE; without it nothing is read or written. Keys name what was
// tuned, the sizes, the precision and the GPU; a later line for the same key replaces an earlier one.
namespace {
std::mutex g_tune_mu;
std::string g_tune_path;
std::map<std::string, std::vector<double>> g_tune;

void tune_load(const std::string& path) {
  g_tune.clear();
  g_tune_path = path;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const std::string kk = "\"key\": \"", vk = "\"values\": [";
    const size_t a = line.find(kk);
    if (a == std::string::npos) continue;
    const size_t b = line.find('"', a + kk.size());
    const size_t c = line.find(vk, b == std::string::npos ? 0 : b);
    if (b == std::string::npos || c == std::string::npos) continue;
    const size_t d = line.find(']', c);
    if (d == std::string::npos) continue;
    std::vector<double> vals;
    const std::string body = line.substr(c + vk.size(), d - c - vk.size());
    size_t pos = 0;
    bool ok = true;
    while (pos < body.size() && ok) {
      size_t e = body.find(',', pos);
      if (e == std::string::npos) e = body.size();
      const std::string tok = body.substr(pos, e - pos);
      char* end = nullptr;
      const double v = std::strtod(tok.c_str(), &end);
      ok = end != tok.c_str();
      if (ok) vals.push_back(v);
      pos = e + 1;
    }
    if (ok) g_tune[line.substr(a + kk.size(), b - a - kk.size())] = vals;
  }
}
}  // namespace

bool tune_cache_get(const std::string& key, std::vector<double>& values) {
  const char* path = std::getenv("TDZ_TUNE_CACHE");
  if (!path || !*path) return false;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (g_tune_path != path) tune_load(path);
  const auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  values = it->second;
  return true;
}

void tune_cache_put(const std::string& key, const std::vector<double>& values) {
  const char* path = std::getenv("TDZ_TUNE_CACHE");
  if (!path || !*path || key.find('"') != std::string::npos) return;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (g_tune_path != path) tune_load(path);
  g_tune[key] = values;
  std::ofstream f(path, std::ios::app);
  if (!f) return;
  f.precision(17);
  f << "{\"key\": \"" << key << "\", \"values\": [";
  for (size_t i = 0; i < values.size(); ++i) f << (i ? ", " : "") << values[i];
  f << "]}\n";
}

// ----------------------------------------------------------------------------- Gauss-Legendre
// Nodes are the roots of P_n, found by Newton's method on the three-term recurrence
// (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, started from the Chebyshev-like guess
// cos(pi (i + 3/4) / (n + 1/2)); weights 2 / ((1 - x^2) P_n'(x)^2).
static double legendre_p(int n, double z, double* pnm1) {
  double pk = z, pkm1 = 1.0;
  for (int k = 1; k < n; ++k) {
    double pkp1 = ((2.0 * k + 1.0) * z * pk - k * pkm1) / (k + 1.0);
    pkm1 = pk;
    pk = pkp1;
  }
  *pnm1 = pkm1;
  return pk;
}

static void legendre_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pnm1 = 0.0, pn = 0.0, dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      pn = legendre_p(n, z, &pnm1);
      dp = n * (pnm1 - z * pn) / (1.0 - z * z);   // (1 - z^2) P_n' = n (P_{n-1} - z P_n)
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    pn = legendre_p(n, z, &pnm1);
    dp = n * (pnm1 - z * pn) / (1.0 - z * z);
    x[n - 1 - i] = z;  // ascending order
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// ----------------------------------------------------------------------------- de Boor
// Values of the p+1 non-zero B-splines on span j at x, by de Boor's triangular scheme
// with the "left/right" distances; also returns the degree p-1 values for derivatives.
static void span_basis(const std::vector<double>& t, int p, int64_t j, double x, double* N, double* dN) {
  double left[16], right[16], tab[17], lower[17];
  tab[0] = 1.0;
  for (int k = 1; k <= p; ++k) {
    if (k == p) std::memcpy(lower, tab, sizeof(double) * p);  // degree p-1 values
    left[k] = x - t[j + 1 - k];
    right[k] = t[j + k] - x;
    double saved = 0.0;
    for (int r = 0; r < k; ++r) {
      double denom = right[r + 1] + left[k - r];
      double temp = denom != 0.0 ? tab[r] / denom : 0.0;
      tab[r] = saved + right[r + 1] * temp;
      saved = left[k - r] * temp;
    }
    tab[k] = saved;
  }
  if (p == 0) {
    N[0] = 1.0;
    dN[0] = 0.0;
    return;
  }
  for (int r = 0; r <= p; ++r) N[r] = tab[r];
  // N'_{i,p} = p/(t_{i+p}-t_i) N_{i,p-1} - p/(t_{i+p+1}-t_{i+1}) N_{i+1,p-1}, i = j-p+r;
  // lower[q] holds N_{j-p+1+q, p-1}
  for (int r = 0; r <= p; ++r) {
    int64_t i = j - p + r;
    double a = (r >= 1) ? lower[r - 1] : 0.0;
    double b = (r <= p - 1) ? lower[r] : 0.0;
    double da = t[i + p] - t[i], db = t[i + p + 1] - t[i + 1];
    dN[r] = (da != 0.0 ? p * a / da : 0.0) - (db != 0.0 ? p * b / db : 0.0);
  }
}

// ----------------------------------------------------------------------------- medium
static int layer_of(const std::vector<double>& b, double x) {
  int nl = (int)b.size() - 1;
  int r = (int)(std::upper_bound(b.begin(), b.end(), x) - b.begin()) - 1;
  return std::min(std::max(r, 0), nl - 1);
}

double Medium::inv_mass(const double* r, int dim) const {
  switch (mass_kind) {
    case TDZ_MASS_CONST: return 1.0 / mass_par[0];
    case TDZ_MASS_QUESNE: return 1.0 + r[0] / mass_par[0];
    case TDZ_MASS_LAYERS: return 1.0 / lmass[layer_of(bounds, r[0])];
    case TDZ_MASS_ELLIPSE: {
      double u = r[0] / mass_par[0], v = dim > 1 ? r[1] / mass_par[1] : 0.0;
      return (u * u + v * v < 1.0) ? 1.0 / mass_par[2] : 1.0 / mass_par[3];
    }
  }
  return 1.0;
}

double Medium::potential(const double* r, int dim) const {
  switch (pot_kind) {
    case TDZ_POT_ZERO: return 0.0;
    case TDZ_POT_SOFTCORE: {
      double s = 0.0;
      for (int a = 0; a < dim; ++a) s += r[a] * r[a];
      return -pot_par[0] / std::sqrt(s + pot_par[1]);
    }
    case TDZ_POT_HO: {
      double s = 0.0;
      for (int a = 0; a < dim; ++a) s += pot_par[a] * pot_par[a] * r[a] * r[a];
      return 0.5 * s;
    }
    case TDZ_POT_QUESNE: {
      double a = pot_par[0], w = pot_par[1], x = r[0];
      return a * w * w * x * x / (8.0 * (x + a));
    }
    case TDZ_POT_LAYERS: return lpot[layer_of(bounds, r[0])];
    case TDZ_POT_ELLIPSE: {
      double u = r[0] / pot_par[0], v = dim > 1 ? r[1] / pot_par[1] : 0.0;
      return (u * u + v * v < 1.0) ? pot_par[2] : pot_par[3];
    }
    case TDZ_POT_H2P: {
      double R = pot_par[0], eps = pot_par[1], x = r[0];
      return -1.0 / std::sqrt((x + 0.5 * R) * (x + 0.5 * R) + eps) - 1.0 / std::sqrt((x - 0.5 * R) * (x - 0.5 * R) + eps);
    }
  }
  return 0.0;
}

double Medium::dpotential(const double* r, int dim, int axis) const {
  switch (pot_kind) {
    case TDZ_POT_SOFTCORE: {
      double s = 0.0;
      for (int a = 0; a < dim; ++a) s += r[a] * r[a];
      double q = s + pot_par[1];
      return pot_par[0] * r[axis] / (q * std::sqrt(q));
    }
    case TDZ_POT_HO: return pot_par[axis] * pot_par[axis] * r[axis];
    case TDZ_POT_QUESNE: {
      double a = pot_par[0], w = pot_par[1], x = r[0];
      return a * w * w * x * (x + 2.0 * a) / (8.0 * (x + a) * (x + a));
    }
    case TDZ_POT_H2P: {
      double R = pot_par[0], eps = pot_par[1], x = r[0];
      double u = x + 0.5 * R, v = x - 0.5 * R;
      double qu = u * u + eps, qv = v * v + eps;
      return u / (qu * std::sqrt(qu)) + v / (qv * std::sqrt(qv));
    }
    default: return 0.0;  // zero, or piecewise constant (gradient zero between interfaces)
  }
}

// 1-D absorbing mask of one coordinate (the layer's definition is in tdz.h, TDZ_CAP_*).
double Medium::cap_axis(double x) const {
  if (cap_kind == TDZ_CAP_NONE) return 0.0;
  const double r0 = cap_par[0], R = cap_par[1];
  const double s = (std::fabs(x) - r0) / (R - r0);
  if (!(s > 0.0)) return 0.0;
  if (cap_kind == TDZ_CAP_POLY) return cap_par[2] * std::pow(s, cap_par[3]);
  // Manolopoulos: (1/(2m)) (2 pi / width)^2 f(c s)
  const double c = 2.62206, c3 = c * c * c;
  const double ca = 1.0 - 16.0 / c3, cb = (1.0 - 17.0 / c3) / (c * c);
  const double y = c * s;
  const double k = 2.0 * M_PI / (R - r0);
  return 0.5 / cap_par[2] * k * k * (ca * y - cb * y * y * y + 4.0 / ((c - y) * (c - y)) - 4.0 / ((c + y) * (c + y)));
}

// ----------------------------------------------------------------------------- 1-D assembly
// One pass over the elements fills all seven band matrices (the fused multi-matrix pass of
// Sec. "Parallel assembly"); Dirichlet end functions are skipped when scattering.
static void assemble_1d(const Basis& B, const Medium& med, Ops& o) {
  const int p = B.p, nq = B.nq, P1 = p + 1;
  const int64_t n = B.nfun - 2;
  Band* mats[] = {&o.S, &o.T, &o.V, &o.H0, &o.D, &o.G, &o.K, &o.W, &o.M};
  for (Band* m : mats) {
    m->n = n;
    m->p = p;
    m->a.assign((size_t)n * P1, 0.0);
  }
  std::vector<double> loc(9 * P1 * P1);
  for (int64_t e = 0; e < B.nelem(); ++e) {
    std::fill(loc.begin(), loc.end(), 0.0);
    for (int q = 0; q < nq; ++q) {
      double x = B.xq[e * nq + q], w = B.wq[e * nq + q];
      double mi = med.inv_mass(&x, 1), v = med.potential(&x, 1), dv = med.dpotential(&x, 1, 0);
      const double eta = med.cap_axis(x);
      const double* N = &B.val[(e * nq + q) * P1];
      const double* dN = &B.der[(e * nq + q) * P1];
      for (int a = 0; a < P1; ++a) {
        for (int c = 0; c <= a; ++c) {
          double nn = w * N[a] * N[c];
          double* L = &loc[a * P1 + c];
          L[0 * P1 * P1] += nn;                           // S
          L[1 * P1 * P1] += 0.5 * w * mi * dN[a] * dN[c];  // T_BDD
          L[2 * P1 * P1] += nn * v;                       // V
          L[4 * P1 * P1] += nn * x;                       // D
          L[5 * P1 * P1] += nn * mi * dv;                 // G
          L[6 * P1 * P1] += nn * mi;                      // K
          L[7 * P1 * P1] += nn * eta;                     // W (absorbing mask)
          L[8 * P1 * P1] += w * mi * (N[a] * dN[c] - dN[a] * N[c]);  // M (velocity, Eq. vel_elem)
        }
      }
    }
    const int64_t first = B.span[e] - p;  // function index of local column 0
    for (int a = 0; a < P1; ++a) {
      for (int c = 0; c <= a; ++c) {
        int64_t fi = first + a, fj = first + c;  // fi >= fj
        if (fj < 1 || fi > B.nfun - 2) continue;
        int64_t i = fi - 1;
        int d = (int)(fi - fj);
        for (int k : {0, 1, 2, 4, 5, 6, 7}) mats[k]->a[(size_t)i * P1 + d] += loc[k * P1 * P1 + a * P1 + c];
        // M is antisymmetric: the local (a, c) entry is M(fi, fj) only when the two local functions map in
        // that order (fi >= fj holds since a >= c and first is common)
        mats[8]->a[(size_t)i * P1 + d] += loc[8 * P1 * P1 + a * P1 + c];
      }
    }
  }
  for (size_t k = 0; k < o.H0.a.size(); ++k) o.H0.a[k] = o.T.a[k] + o.V.a[k];
}

// ----------------------------------------------------------------------------- 2-D / 3-D factors
// Per-axis 1-D bands of the tensor-product basis (Eq. tensor3d): S_a, the unit-mass kinetic factor
// T1_a = 1/2 <N'|N'> and the dipole factor D_a, by the same element quadrature as in 1-D. The
// non-separable potential and mass are applied on the GPU at the Gauss points of the same tables.
static void assemble_axis(const Basis& B, const Medium& med, Band& S, Band& T1, Band& D, Band& Wm) {
  const int p = B.p, nq = B.nq, P1 = p + 1;
  const int64_t n = B.nfun - 2;
  for (Band* m : {&S, &T1, &D, &Wm}) {
    m->n = n;
    m->p = p;
    m->a.assign((size_t)n * P1, 0.0);
  }
  for (int64_t e = 0; e < B.nelem(); ++e) {
    const int64_t first = B.span[e] - p;
    for (int a = 0; a < P1; ++a)
      for (int c = 0; c <= a; ++c) {
        const int64_t fi = first + a, fj = first + c;
        if (fj < 1 || fi > B.nfun - 2) continue;
        double s = 0, t = 0, d = 0, wm = 0;
        for (int q = 0; q < nq; ++q) {
          const double w = B.wq[e * nq + q], x = B.xq[e * nq + q];
          const double* N = &B.val[(e * nq + q) * P1];
          const double* dN = &B.der[(e * nq + q) * P1];
          s += w * N[a] * N[c];
          t += 0.5 * w * dN[a] * dN[c];
          d += w * x * N[a] * N[c];
          wm += w * med.cap_axis(x) * N[a] * N[c];
        }
        const size_t k = (size_t)(fi - 1) * P1 + (fi - fj);
        S.a[k] += s;
        T1.a[k] += t;
        D.a[k] += d;
        Wm.a[k] += wm;
      }
  }
}

// ----------------------------------------------------------------------------- ground state
// Real symmetric band LDL^T (no pivoting; used for H0 - sigma S with sigma below the spectrum,
// which is positive definite) and the matching solve.
static bool band_ldlt(std::vector<double>& a, int64_t n, int p) {
  const int P1 = p + 1;
  double l[17];
  for (int64_t j = 0; j < n; ++j) {
    // a[j][0] holds the pivot after the updates of earlier columns (right-looking)
    double dj = a[j * P1];
    if (!(std::fabs(dj) > 0.0)) return false;
    int rmax = (int)std::min<int64_t>(p, n - 1 - j);
    for (int r = 1; r <= rmax; ++r) l[r] = a[(j + r) * P1 + r] / dj;
    for (int r = 1; r <= rmax; ++r) {
      for (int c = 1; c <= r; ++c) a[(j + r) * P1 + (r - c)] -= l[r] * l[c] * dj;  // entry (j+r, j+c)
      a[(j + r) * P1 + r] = l[r];                                                 // L(j+r, j)
    }
  }
  return true;
}

static void band_ldlt_solve(const std::vector<double>& f, int64_t n, int p, std::vector<double>& x) {
  const int P1 = p + 1;
  for (int64_t i = 0; i < n; ++i) {
    double s = x[i];
    for (int d = 1; d <= p && d <= i; ++d) s -= f[i * P1 + d] * x[i - d];
    x[i] = s;
  }
  for (int64_t i = 0; i < n; ++i) x[i] /= f[i * P1];
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int d = 1; d <= p && i + d < n; ++d) s -= f[(i + d) * P1 + d] * x[i + d];
    x[i] = s;
  }
}

static void band_matvec(const Band& M, const std::vector<double>& x, std::vector<double>& y) {
  const int64_t n = M.n;
  const int p = M.p;
  for (int64_t i = 0; i < n; ++i) {
    double s = M.at(i, 0) * x[i];
    for (int d = 1; d <= p; ++d) {
      if (i - d >= 0) s += M.at(i, d) * x[i - d];
      if (i + d < n) s += M.at(i + d, d) * x[i + d];
    }
    y[i] = s;
  }
}

}  // namespace tdz

using namespace tdz;

// ============================================================================= C ABI
extern "C" {

const char* tdz_last_error(void) { return g_err.c_str(); }

int tdz_basis_create(const double* knots, int64_t nknots, int degree, int nquad, tdz_basis** out) {
  if (!knots || !out || degree < 1 || degree > 8 || nquad < 1 || nquad > 16 || nknots < 2 * (degree + 1)) {
    set_error("tdz_basis_create: bad arguments (degree 1..8, nquad 1..16, nknots >= 2(degree+1))");
    return TDZ_EINVAL;
  }
  for (int64_t i = 1; i < nknots; ++i)
    if (!(knots[i] >= knots[i - 1]) || !std::isfinite(knots[i])) {
      set_error("tdz_basis_create: knots must be finite and non-decreasing");
      return TDZ_EINVAL;
    }
  for (int k = 1; k <= degree; ++k)
    if (knots[k] != knots[0] || knots[nknots - 1 - k] != knots[nknots - 1]) {
      set_error("tdz_basis_create: knot vector is not open (ends must repeat degree+1 times)");
      return TDZ_EINVAL;
    }
  tdz_basis* h = new (std::nothrow) tdz_basis;
  if (!h) return TDZ_ENOMEM;
  Basis& B = h->b;
  B.knots.assign(knots, knots + nknots);
  B.p = degree;
  B.nq = nquad;
  B.nfun = nknots - degree - 1;
  std::vector<double> gx, gw;
  legendre_rule(nquad, gx, gw);
  for (int64_t j = degree; j < B.nfun; ++j)
    if (B.knots[j + 1] > B.knots[j]) B.span.push_back(j);
  if (B.span.empty() || B.nfun < 3) {
    delete h;
    set_error("tdz_basis_create: no non-empty span or fewer than 3 functions");
    return TDZ_EINVAL;
  }
  const int P1 = degree + 1;
  const int64_t E = B.nelem();
  B.xq.resize(E * nquad);
  B.wq.resize(E * nquad);
  B.val.resize(E * nquad * P1);
  B.der.resize(E * nquad * P1);
  for (int64_t e = 0; e < E; ++e) {
    int64_t j = B.span[e];
    double a = B.knots[j], b = B.knots[j + 1], h2 = 0.5 * (b - a), m = 0.5 * (a + b);
    for (int q = 0; q < nquad; ++q) {
      double x = m + h2 * gx[q];
      B.xq[e * nquad + q] = x;
      B.wq[e * nquad + q] = h2 * gw[q];
      span_basis(B.knots, degree, j, x, &B.val[(e * nquad + q) * P1], &B.der[(e * nquad + q) * P1]);
    }
  }
  *out = h;
  return TDZ_OK;
}

int tdz_basis_info(const tdz_basis* b, int64_t* nfun, int64_t* nelem, int* degree, int* nquad) {
  if (!b) return TDZ_EINVAL;
  if (nfun) *nfun = b->b.nfun;
  if (nelem) *nelem = b->b.nelem();
  if (degree) *degree = b->b.p;
  if (nquad) *nquad = b->b.nq;
  return TDZ_OK;
}

int tdz_basis_eval(const tdz_basis* bh, const double* x, int64_t npts, double* val, double* der) {
  if (!bh || !x || !val || !der || npts < 0) return TDZ_EINVAL;
  const Basis& B = bh->b;
  const int p = B.p;
  std::memset(val, 0, sizeof(double) * B.nfun * npts);
  std::memset(der, 0, sizeof(double) * B.nfun * npts);
  double N[17], dN[17];
  for (int64_t k = 0; k < npts; ++k) {
    // last span whose left knot is <= x (right end point belongs to the last span)
    int64_t lo = 0, hi = B.nelem() - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) / 2;
      if (B.knots[B.span[mid]] <= x[k]) lo = mid; else hi = mid - 1;
    }
    int64_t j = B.span[lo];
    span_basis(B.knots, p, j, x[k], N, dN);
    for (int r = 0; r <= p; ++r) {
      val[(j - p + r) * npts + k] = N[r];
      der[(j - p + r) * npts + k] = dN[r];
    }
  }
  return TDZ_OK;
}

void tdz_basis_destroy(tdz_basis* b) { delete b; }

int tdz_assemble(const tdz_basis* const* axes, int dim, const tdz_medium* medium, tdz_ops** out) {
  if (!axes || !medium || !out || dim < 1 || dim > 3) return TDZ_EINVAL;
  for (int a = 0; a < dim; ++a)
    if (!axes[a]) return TDZ_EINVAL;
  if (dim > 1) {
    for (int a = 0; a < dim; ++a) {
      const Basis& B = axes[a]->b;
      if (B.p != axes[0]->b.p) {
        set_error("tdz_assemble: all axes must have the same degree");
        return TDZ_EUNSUPPORTED;
      }
      for (int64_t e = 0; e < B.nelem(); ++e)
        if (B.span[e] != e + B.p) {
          set_error("tdz_assemble: 2-D/3-D needs distinct interior knots (one element per span)");
          return TDZ_EUNSUPPORTED;
        }
    }
  }
  Medium med;
  med.mass_kind = medium->mass_kind;
  med.pot_kind = medium->pot_kind;
  std::memcpy(med.mass_par, medium->mass_par, sizeof(med.mass_par));
  std::memcpy(med.pot_par, medium->pot_par, sizeof(med.pot_par));
  if (med.mass_kind < 0 || med.mass_kind > 3 || med.pot_kind < 0 || med.pot_kind > 6) {
    set_error("tdz_assemble: unknown mass or potential kind");
    return TDZ_EINVAL;
  }
  if (med.mass_kind == TDZ_MASS_LAYERS || med.pot_kind == TDZ_POT_LAYERS) {
    if (medium->nlayers < 1 || !medium->layer_bounds) return TDZ_EINVAL;
    med.bounds.assign(medium->layer_bounds, medium->layer_bounds + medium->nlayers + 1);
    if (med.mass_kind == TDZ_MASS_LAYERS) {
      if (!medium->layer_mass) return TDZ_EINVAL;
      med.lmass.assign(medium->layer_mass, medium->layer_mass + medium->nlayers);
      for (double m : med.lmass)
        if (!(m > 0)) return TDZ_EINVAL;
    }
    if (med.pot_kind == TDZ_POT_LAYERS) {
      if (!medium->layer_pot) return TDZ_EINVAL;
      med.lpot.assign(medium->layer_pot, medium->layer_pot + medium->nlayers);
    }
  }
  if (med.mass_kind == TDZ_MASS_CONST && !(med.mass_par[0] > 0)) return TDZ_EINVAL;
  med.cap_kind = medium->cap_kind;
  std::memcpy(med.cap_par, medium->cap_par, sizeof(med.cap_par));
  if (med.cap_kind < TDZ_CAP_NONE || med.cap_kind > TDZ_CAP_MANOLOPOULOS) {
    set_error("tdz_assemble: unknown absorbing-layer kind");
    return TDZ_EINVAL;
  }
  if (med.cap_kind != TDZ_CAP_NONE) {
    const double r0 = med.cap_par[0], R = med.cap_par[1];
    bool ok = r0 >= 0.0 && R > r0 && std::isfinite(R);
    if (med.cap_kind == TDZ_CAP_POLY) ok = ok && med.cap_par[2] >= 0.0 && med.cap_par[3] >= 0.0;
    if (med.cap_kind == TDZ_CAP_MANOLOPOULOS) {
      ok = ok && med.cap_par[2] > 0.0;
      // the mask diverges at |x_a| = R: no quadrature point may reach it (R at or beyond the domain's edge)
      for (int a = 0; a < dim && ok; ++a)
        for (double x : axes[a]->b.xq) ok = ok && std::fabs(x) < R;
    }
    if (!ok) {
      set_error("tdz_assemble: invalid absorbing-layer parameters (0 <= r0 < R; eta0, k >= 0; m > 0; the "
                "Manolopoulos layer must end at or beyond the domain's edge)");
      return TDZ_EINVAL;
    }
  }
  if (dim > 1 && (med.mass_kind == TDZ_MASS_LAYERS || med.mass_kind == TDZ_MASS_QUESNE ||
                  med.pot_kind == TDZ_POT_LAYERS || med.pot_kind == TDZ_POT_QUESNE || med.pot_kind == TDZ_POT_H2P)) {
    set_error("tdz_assemble: 1-D-only medium kind in a 2-D/3-D assembly");
    return TDZ_EINVAL;
  }
  tdz_ops* h = new (std::nothrow) tdz_ops;
  if (!h) return TDZ_ENOMEM;
  Ops& o = h->o;
  o.dim = dim;
  o.med = med;
  try {
    for (int a = 0; a < dim; ++a) {
      o.n[a] = axes[a]->b.nfun - 2;
      o.p[a] = axes[a]->b.p;
    }
    if (dim == 1) {
      assemble_1d(axes[0]->b, med, o);
    } else {
      for (int a = 0; a < dim; ++a) {
        o.axis[a] = axes[a]->b;
        assemble_axis(o.axis[a], med, o.Sa[a], o.T1a[a], o.Da[a], o.Wa[a]);
      }
    }
  } catch (const std::bad_alloc&) {
    delete h;
    return TDZ_ENOMEM;
  }
  *out = h;
  return TDZ_OK;
}

int tdz_ops_info(const tdz_ops* ops, int* dim, int64_t* shape, int* degree) {
  if (!ops) return TDZ_EINVAL;
  if (dim) *dim = ops->o.dim;
  for (int a = 0; a < ops->o.dim; ++a) {
    if (shape) shape[a] = ops->o.n[a];
    if (degree) degree[a] = ops->o.p[a];
  }
  return TDZ_OK;
}

int tdz_ops_band(const tdz_ops* ops, int which, int axis, double* out) {
  if (!ops || !out || axis < 0 || axis >= ops->o.dim) return TDZ_EINVAL;
  const Band* m = nullptr;
  if (ops->o.dim > 1) {
    switch (which) {
      case TDZ_MAT_S: m = &ops->o.Sa[axis]; break;
      case TDZ_MAT_T: m = &ops->o.T1a[axis]; break;
      case TDZ_MAT_D: m = &ops->o.Da[axis]; break;
      case TDZ_MAT_W: m = &ops->o.Wa[axis]; break;
      default:
        set_error("tdz_ops_band: 2-D/3-D operators expose the per-axis S, T (unit mass), D and W factors");
        return TDZ_EINVAL;
    }
    std::memcpy(out, m->a.data(), sizeof(double) * m->a.size());
    return TDZ_OK;
  }
  switch (which) {
    case TDZ_MAT_S: m = &ops->o.S; break;
    case TDZ_MAT_T: m = &ops->o.T; break;
    case TDZ_MAT_V: m = &ops->o.V; break;
    case TDZ_MAT_H0: m = &ops->o.H0; break;
    case TDZ_MAT_D: m = &ops->o.D; break;
    case TDZ_MAT_G: m = &ops->o.G; break;
    case TDZ_MAT_K: m = &ops->o.K; break;
    case TDZ_MAT_W: m = &ops->o.W; break;
    case TDZ_MAT_VEL: m = &ops->o.M; break;
    default: return TDZ_EINVAL;
  }
  std::memcpy(out, m->a.data(), sizeof(double) * m->a.size());
  return TDZ_OK;
}

void tdz_ops_destroy(tdz_ops* ops) { delete ops; }

int tdz_ground_state(const tdz_ops* ops, double* energy, double* c) {
  if (!ops || !energy || !c || ops->o.dim != 1) return TDZ_EINVAL;
  const Ops& o = ops->o;
  const int64_t n = o.S.n;
  const int p = o.S.p, P1 = p + 1;
  // shift below the spectrum: the potential minimum over the diagonal Rayleigh quotients
  double vmin = 1e300;
  for (int64_t i = 0; i < n; ++i) vmin = std::min(vmin, o.V.at(i, 0) / o.S.at(i, 0));
  double sigma = vmin - 0.05 * (1.0 + std::fabs(vmin));
  std::vector<double> f(o.H0.a.size());
  for (size_t k = 0; k < f.size(); ++k) f[k] = o.H0.a[k] - sigma * o.S.a[k];
  if (!band_ldlt(f, n, p)) {
    set_error("tdz_ground_state: factorisation failed");
    return TDZ_ENOCONV;
  }
  std::vector<double> x(n, 1.0), y(n), sx(n), hx(n);
  double lam = 0.0;
  bool ok = false;
  for (int it = 0; it < 20000; ++it) {
    band_matvec(o.S, x, y);
    band_ldlt_solve(f, n, p, y);
    band_matvec(o.S, y, sx);
    band_matvec(o.H0, y, hx);
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      num += y[i] * hx[i];
      den += y[i] * sx[i];
    }
    lam = num / den;
    // normalise with the sign of the largest component fixed, then measure the change
    double s = 1.0 / std::sqrt(den);
    int64_t im = 0;
    for (int64_t i = 0; i < n; ++i)
      if (std::fabs(y[i]) > std::fabs(y[im])) im = i;
    if (y[im] < 0) s = -s;
    double dx = 0.0, xx = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double v = y[i] * s;
      dx = std::max(dx, std::fabs(v - x[i]));
      xx = std::max(xx, std::fabs(v));
      x[i] = v;
    }
    if (it > 3 && dx <= 4e-16 * xx) {
      ok = true;
      break;
    }
  }
  (void)P1;
  int64_t imax = 0;
  for (int64_t i = 0; i < n; ++i)
    if (std::fabs(x[i]) > std::fabs(x[imax])) imax = i;
  double sgn = x[imax] < 0 ? -1.0 : 1.0;
  for (int64_t i = 0; i < n; ++i) {
    c[2 * i] = sgn * x[i];
    c[2 * i + 1] = 0.0;
  }
  *energy = lam;
  if (!ok) {
    set_error("tdz_ground_state: inverse iteration did not settle");
    return TDZ_ENOCONV;
  }
  return TDZ_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------- a_Q
// The position-dependent-mass term of the dipole acceleration (Eq. aQ_definition) in 1-D: (i/4) <[p m^-1 p,
// p m^-1 + m^-1 p]> = i <[T, v]>; in the Galerkin basis an operator product A B is A S^-1 B, so
// a_Q = i c^H (T S^-1 Vel - Vel S^-1 T) c = -2 Im[(T c)^H S^-1 (Vel c)], with Vel = -(i/2) M.
// S is factored once (real symmetric positive definite band, LDL^T) and reused for every state.
extern "C" int tdz_pdm_acceleration(const tdz_ops* ops, const double* c, int64_t nstates, double* aq) {
  if (!ops || !c || !aq || nstates < 1 || ops->o.dim != 1) return TDZ_EINVAL;
  const Ops& o = ops->o;
  const int64_t n = o.S.n;
  const int p = o.S.p, P1 = p + 1;
  std::vector<double> f(o.S.a);
  if (!band_ldlt(f, n, p)) {
    set_error("tdz_pdm_acceleration: overlap factorisation failed");
    return TDZ_ENOCONV;
  }
  std::vector<double> cr(n), ci(n), tr(n), ti(n), vr(n), vi(n);
  for (int64_t s = 0; s < nstates; ++s) {
    const double* x = c + 2 * n * s;
    for (int64_t i = 0; i < n; ++i) {
      cr[i] = x[2 * i];
      ci[i] = x[2 * i + 1];
    }
    band_matvec(o.T, cr, tr);
    band_matvec(o.T, ci, ti);
    // M c with M antisymmetric: row i sums M(i, i-d) c_{i-d} - M(i+d, i) c_{i+d}
    for (int64_t i = 0; i < n; ++i) {
      double ar = 0.0, ai = 0.0;
      for (int d = 1; d <= p; ++d) {
        if (i - d >= 0) {
          ar += o.M.a[(size_t)i * P1 + d] * cr[i - d];
          ai += o.M.a[(size_t)i * P1 + d] * ci[i - d];
        }
        if (i + d < n) {
          ar -= o.M.a[(size_t)(i + d) * P1 + d] * cr[i + d];
          ai -= o.M.a[(size_t)(i + d) * P1 + d] * ci[i + d];
        }
      }
      // Vel c = -(i/2) M c
      vr[i] = 0.5 * ai;
      vi[i] = -0.5 * ar;
    }
    band_ldlt_solve(f, n, p, vr);
    band_ldlt_solve(f, n, p, vi);
    // z = (T c)^H x = sum conj(t_i) x_i; a_Q = -2 Im z
    double zi = 0.0;
    for (int64_t i = 0; i < n; ++i) zi += tr[i] * vi[i] - ti[i] * vr[i];
    aq[s] = -2.0 * zi;
  }
  return TDZ_OK;
}

// ----------------------------------------------------------------------------- populations and currents
// Projections of 1-D states on nev field-free eigenstates phi_n (Sec. "Currents and coherence dynamics"):
// c_n = phi_n^H S c, the populations |c_n|^2, and the decomposition of the total dipole velocity
// J_tot = c^H Vel c into J_intra = sum_n |c_n|^2 v_nn, J_inter = sum_{m != n} conj(c_m) c_n v_mn (v_mn =
// phi_m^H Vel phi_n, Vel = -(i/2) M) and the remainder J_bc = J_tot - J_intra - J_inter (Eqs.
// Jdecomp-Jbc).
extern "C" int tdz_populations(const tdz_ops* ops, const double* phi, int nev, const double* c, int64_t nstates,
                               double* pop, double* jdec) {
  if (!ops || !phi || !c || nev < 1 || nstates < 1 || ops->o.dim != 1 || (!pop && !jdec)) return TDZ_EINVAL;
  const Ops& o = ops->o;
  const int64_t n = o.S.n;
  const int p = o.S.p, P1 = p + 1;
  using cd = std::complex<double>;
  auto load = [&](const double* x, std::vector<cd>& v) {
    v.resize(n);
    for (int64_t i = 0; i < n; ++i) v[i] = cd(x[2 * i], x[2 * i + 1]);
  };
  auto band = [&](const Band& B, const std::vector<cd>& x, std::vector<cd>& y) {  // symmetric band
    y.assign(n, cd(0.0, 0.0));
    for (int64_t i = 0; i < n; ++i) {
      cd s = B.at(i, 0) * x[i];
      for (int d = 1; d <= p; ++d) {
        if (i - d >= 0) s += B.at(i, d) * x[i - d];
        if (i + d < n) s += B.at(i + d, d) * x[i + d];
      }
      y[i] = s;
    }
  };
  auto vel = [&](const std::vector<cd>& x, std::vector<cd>& y) {  // Vel x = -(i/2) M x, M antisymmetric
    y.assign(n, cd(0.0, 0.0));
    for (int64_t i = 0; i < n; ++i) {
      cd s(0.0, 0.0);
      for (int d = 1; d <= p; ++d) {
        if (i - d >= 0) s += o.M.a[(size_t)i * P1 + d] * x[i - d];
        if (i + d < n) s -= o.M.a[(size_t)(i + d) * P1 + d] * x[i + d];
      }
      y[i] = cd(0.0, -0.5) * s;
    }
  };
  auto dotc = [&](const std::vector<cd>& a, const std::vector<cd>& b) {
    cd s(0.0, 0.0);
    for (int64_t i = 0; i < n; ++i) s += std::conj(a[i]) * b[i];
    return s;
  };
  std::vector<std::vector<cd>> ph(nev), vph(nev);
  for (int k = 0; k < nev; ++k) {
    load(phi + 2 * n * k, ph[k]);
    vel(ph[k], vph[k]);
  }
  std::vector<cd> vmn((size_t)nev * nev);
  for (int m = 0; m < nev; ++m)
    for (int k = 0; k < nev; ++k) vmn[(size_t)m * nev + k] = dotc(ph[m], vph[k]);
  std::vector<cd> x, sx, vx;
  std::vector<cd> cn(nev);
  for (int64_t s = 0; s < nstates; ++s) {
    load(c + 2 * n * s, x);
    band(o.S, x, sx);
    for (int k = 0; k < nev; ++k) {
      cn[k] = dotc(ph[k], sx);
      if (pop) pop[s * nev + k] = std::norm(cn[k]);
    }
    if (jdec) {
      vel(x, vx);
      const double jt = std::real(dotc(x, vx));
      double ji = 0.0, je = 0.0;
      for (int m = 0; m < nev; ++m)
        for (int k = 0; k < nev; ++k) {
          const double t = std::real(std::conj(cn[m]) * cn[k] * vmn[(size_t)m * nev + k]);
          if (m == k) ji += t;
          else je += t;
        }
      jdec[4 * s + 0] = jt;
      jdec[4 * s + 1] = ji;
      jdec[4 * s + 2] = je;
      jdec[4 * s + 3] = jt - ji - je;
    }
  }
  return TDZ_OK;
}
