// Harmonic spectrum of the per-step observables (Sec. "Dipoles"): the Kaiser-windowed Fourier transform
//     F(w) = dt sum_k s(t_k) W_k e^{i w t_k},   t_k = k dt,   S(w) = |F(w)|^2  (times w^4 for the length
// form, which turns a dipole record into the acceleration spectrum), and the yield of each odd harmonic
// (the integral of S over [(q - 1/2) w0, (q + 1/2) w0], trapezoid rule on the frequency grid).
//
// The transform is a direct sum in binary64 at the caller's frequencies (the spectrum of a strong-field
// record spans many decades, and the weak plateau harmonics sit on the large fundamental, so the sums
// need the 53-bit significand). One thread per frequency; a block's threads share tiles of the windowed
// record in shared memory; e^{i w t_k} advances by the rotation e^{i w dt} inside a tile and is recomputed
// exactly at every tile start.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "tdz_internal.h"

namespace tdz {
namespace {

constexpr int kSpecThreads = 128;
constexpr int kSpecTile = 256;

__global__ void k_spectrum(const double* __restrict__ sig, long long nt, long long sig_stride, long long t_stride,
                           const double* __restrict__ win, double dt, double w_lo, double dw, long long nw,
                           int length_form, double* __restrict__ S) {
  __shared__ double tile[kSpecTile];
  const long long s = blockIdx.y;
  const long long j = (long long)blockIdx.x * kSpecThreads + threadIdx.x;
  const double w = w_lo + (double)j * dw;
  const double* x = sig + s * sig_stride;
  double fr = 0.0, fi = 0.0;
  double cr = 1.0, ci = 0.0, rr = 1.0, ri = 0.0;
  sincos(w * dt, &ri, &rr);  // rotation e^{i w dt}
  for (long long k0 = 0; k0 < nt; k0 += kSpecTile) {
    __syncthreads();
    for (int t = threadIdx.x; t < kSpecTile; t += kSpecThreads) {
      const long long k = k0 + t;
      tile[t] = k < nt ? x[k * t_stride] * win[k] : 0.0;
    }
    __syncthreads();
    sincos(w * (double)k0 * dt, &ci, &cr);  // e^{i w t_k0}, exact at the tile start
    const int n = (int)((nt - k0) < kSpecTile ? (nt - k0) : kSpecTile);
    for (int t = 0; t < n; ++t) {
      const double v = tile[t];
      fr = fma(v, cr, fr);
      fi = fma(v, ci, fi);
      const double nr = cr * rr - ci * ri;
      ci = fma(cr, ri, ci * rr);
      cr = nr;
    }
  }
  if (j < nw) {
    double p = (fr * fr + fi * fi) * dt * dt;
    if (length_form) p *= (w * w) * (w * w);
    S[s * nw + j] = p;
  }
}

// Modified Bessel function I0 by its power series, sum_m ((x/2)^m / m!)^2 (all terms positive).
double bessel_i0(double x) {
  const double q = 0.25 * x * x;
  double term = 1.0, sum = 1.0;
  for (int m = 1; m < 500; ++m) {
    term *= q / ((double)m * (double)m);
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return TDZ_ECUDA;
}

}  // namespace
}  // namespace tdz

using namespace tdz;

extern "C" int tdz_spectrum(const double* signal, int64_t nsig, int64_t nt, int64_t sig_stride, int64_t t_stride,
                            double dt, double beta, int length_form, double w_lo, double dw, int64_t nw, double* S,
                            void* cuda_stream) {
  if (!signal || !S || nsig < 1 || nt < 2 || nw < 1 || t_stride < 1 || sig_stride < 0 || !(dt > 0) ||
      !std::isfinite(dt) || !(beta >= 0) || !std::isfinite(w_lo) || !std::isfinite(dw) || nsig > 65535) {
    set_error("tdz_spectrum: bad arguments");
    return TDZ_EINVAL;
  }
  if (sig_stride == 0 && nsig > 1) {
    set_error("tdz_spectrum: sig_stride 0 with several signals");
    return TDZ_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // Kaiser window, W_k = I0(beta sqrt(1 - (2k/(nt-1) - 1)^2)) / I0(beta)
  std::vector<double> win((size_t)nt);
  const double i0b = bessel_i0(beta);
  for (int64_t k = 0; k < nt; ++k) {
    const double u = 2.0 * (double)k / (double)(nt - 1) - 1.0;
    win[(size_t)k] = bessel_i0(beta * std::sqrt(std::fmax(0.0, 1.0 - u * u))) / i0b;
  }
  const size_t sig_elems = (size_t)((nsig - 1) * sig_stride + (nt - 1) * t_stride + 1);
  const bool dev_in = on_device(signal), dev_out = on_device(S);
  double *d_win = nullptr, *d_sig = nullptr, *d_S = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d_win), sizeof(double) * nt, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_win, win.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, st);
  const double* src = signal;
  if (e == cudaSuccess && !dev_in) {
    e = cudaMallocAsync(reinterpret_cast<void**>(&d_sig), sizeof(double) * sig_elems, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_sig, signal, sizeof(double) * sig_elems, cudaMemcpyHostToDevice, st);
    src = d_sig;
  }
  double* dst = S;
  if (e == cudaSuccess && !dev_out) {
    e = cudaMallocAsync(reinterpret_cast<void**>(&d_S), sizeof(double) * nsig * nw, st);
    dst = d_S;
  }
  if (e == cudaSuccess) {
    const dim3 grid((unsigned)((nw + kSpecThreads - 1) / kSpecThreads), (unsigned)nsig);
    k_spectrum<<<grid, kSpecThreads, 0, st>>>(src, nt, sig_stride, t_stride, d_win, dt, w_lo, dw, nw, length_form, dst);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !dev_out)
    e = cudaMemcpyAsync(S, d_S, sizeof(double) * nsig * nw, cudaMemcpyDeviceToHost, st);
  if (d_win) cudaFreeAsync(d_win, st);
  if (d_sig) cudaFreeAsync(d_sig, st);
  if (d_S) cudaFreeAsync(d_S, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e, "tdz_spectrum");
  return TDZ_OK;
}

extern "C" int tdz_harmonic_yields(const double* S, int64_t nsig, double w_lo, double dw, int64_t nw, double omega0,
                                   int qmax, double* Y) {
  if (!S || !Y || nsig < 1 || nw < 1 || !(dw > 0) || !(omega0 > 0) || qmax < 1) {
    set_error("tdz_harmonic_yields: bad arguments");
    return TDZ_EINVAL;
  }
  const int nq = (qmax + 1) / 2;
  for (int64_t s = 0; s < nsig; ++s) {
    const double* row = S + s * nw;
    for (int h = 0; h < nq; ++h) {
      const int q = 2 * h + 1;
      const double a = (q - 0.5) * omega0, b = (q + 0.5) * omega0;
      // grid points inside [a, b]: j with a <= w_lo + j dw <= b
      int64_t j0 = (int64_t)std::ceil((a - w_lo) / dw), j1 = (int64_t)std::floor((b - w_lo) / dw);
      while (j0 > 0 && w_lo + (double)(j0 - 1) * dw >= a) --j0;
      while (w_lo + (double)j0 * dw < a) ++j0;
      while (w_lo + (double)(j1 + 1) * dw <= b) ++j1;
      while (j1 >= j0 && w_lo + (double)j1 * dw > b) --j1;
      j0 = std::max<int64_t>(j0, 0);
      j1 = std::min<int64_t>(j1, nw - 1);
      double y = 0.0;
      for (int64_t j = j0; j < j1; ++j) y += 0.5 * dw * (row[j] + row[j + 1]);
      Y[s * nq + h] = y;
    }
  }
  return TDZ_OK;
}
