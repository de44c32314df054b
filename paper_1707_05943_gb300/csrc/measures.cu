// measures.cu -- readouts derived from the march: the two-photon wavefunction
// chi of Eq. 2 (FDTD_READ_CHI, below), and the non-Markovian measures of
// App. D on the snapshot rows of a stimulated-emission march
// (FDTD_READ_MEASURES):
//   mu(t)     = int phi*(x,t) psi(x,t) dx,
//   lambda(t) = int |psi(x,t)|^2 dx - |e0(t)|^2,
//   det M_t   = |mu(t)|^2 lambda(t),
// with phi(x,t) the photon of the one-excitation sector (atom starting in its
// ground state, the same packet phi0 incident), the free packet minus the
// emission of the atom at x = -a and of its mirror image at x = +a:
//   phi(x,t) = phi0(x-t) - sqrt(Gamma/2) [ theta(x+a) theta(t-x-a) e0(t-x-a)
//                                         - theta(x-a) theta(t-x+a) e0(t-x+a) ],
// theta(0) = 1/2.  On the grid (column m, row n, r2 = n - m - D/2) the
// retarded times are r2 delta and (r2 + D) delta, so every term is a table
// entry.  x <= -a is exact (psi = phi0(x-t) e1(t), phi = phi0(x-t), and
// int_{-inf}^{-a} |phi0(x-t)|^2 dx = e^{-alpha Gamma t}); x > -a is the
// trapezoid over [-a, x_last], first node psi(-a,t) with the right limit of
// phi.  FP64 throughout; one block per snapshot row, a fixed reduction order.
#include <cuda_runtime.h>

#include "fdtd_internal.cuh"

namespace fdtd {

namespace {
constexpr int kMeasThreads = 256;

__device__ __forceinline__ cd conjm(cd a, cd b) {  // conj(a) * b
  return cd{a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

__global__ void __launch_bounds__(kMeasThreads) k_measures(const cd* __restrict__ snaps, int64_t nx, int tstep,
                                                           const cd* __restrict__ e1tab,
                                                           const cd* __restrict__ e0tab,
                                                           const cd* __restrict__ phitab,
                                                           const double* __restrict__ norms, int D, double delta,
                                                           double gamma, double alpha, double* __restrict__ out) {
  __shared__ double s_re[kMeasThreads], s_im[kMeasThreads];
  const int64_t srow = blockIdx.x;
  const int64_t n = srow * (int64_t)(tstep + 1);
  const int Dh = D / 2;
  const double g = sqrt(0.5 * gamma);
  const cd* row = snaps + srow * nx;
  double are = 0.0, aim = 0.0;
  for (int64_t j = threadIdx.x; j < nx; j += kMeasThreads) {
    const int64_t m = j - Dh + 1;
    const int64_t r2 = n - j - 1;  // (t - x - a) / delta
    cd ph = (r2 >= 0) ? phitab[r2] : cd{0.0, 0.0};
    if (r2 >= 0) ph = ph - (r2 == 0 ? 0.5 * g : g) * e0tab[r2];
    const int64_t r3 = r2 + D;  // (t - x + a) / delta
    if (m >= Dh && r3 >= 0) {
      const double w = (m == Dh ? 0.5 : 1.0) * (r3 == 0 ? 0.5 : 1.0);
      ph = ph + (w * g) * e0tab[r3];
    }
    cd v = conjm(ph, row[j]);
    if (j == nx - 1) v = 0.5 * v;
    are += v.re;
    aim += v.im;
  }
  s_re[threadIdx.x] = are;
  s_im[threadIdx.x] = aim;
  __syncthreads();
  for (int o = kMeasThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_re[threadIdx.x] += s_re[threadIdx.x + o];
      s_im[threadIdx.x] += s_im[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const cd e1 = e1tab[n], e0 = e0tab[n];
    // first node x = -a: psi(-a,t) = phi0(-a-t) e1(t), phi's right limit
    const cd phl = phitab[n] - (n == 0 ? 0.5 * g : g) * e0;
    const cd v0 = conjm(phl, phitab[n] * e1);
    const double acc_re = 0.5 * v0.re + s_re[0], acc_im = 0.5 * v0.im + s_im[0];
    const double decay = exp(-alpha * gamma * n * delta);
    const double mre = e1.re * decay + delta * acc_re, mim = e1.im * decay + delta * acc_im;
    const double lam = cabs2(e1) * decay + norms[n] - cabs2(e0);
    out[4 * srow] = mre;
    out[4 * srow + 1] = mim;
    out[4 * srow + 2] = lam;
    out[4 * srow + 3] = (mre * mre + mim * mim) * lam;
  }
}
}  // namespace

// chi(x1, x2, t) of Eq. 2 from the probes and the exact boundary, one thread per point
__global__ void k_chi(const ChiRec* __restrict__ recs, int64_t count, const double2* __restrict__ probe_val,
                      const cd* __restrict__ phitab, const cd* __restrict__ etab, const cd* __restrict__ phitab2,
                      const cd* __restrict__ etab2, double C, double gamma, int incident,
                      double2* __restrict__ out) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= count) return;
  const ChiRec& r = recs[q];
  cd sum = cd{0.0, 0.0};
  for (int t = 0; t < 4; ++t) {
    cd v = cd{0.0, 0.0};
    if (r.kind[t] == 1) {
      const double2 p = probe_val[r.idx[t]];
      v = cd{p.x, p.y};
    } else if (r.kind[t] == 2) {
      v = phitab[r.idx[t]] * etab[r.row[t]];
      if (phitab2) v = v + phitab2[r.idx[t]] * etab2[r.row[t]];  // second photon of a pair
      v = C * v;
    }
    sum = sum + r.w[t] * v;
  }
  cd c0 = cd{0.0, 0.0};
  if (incident && r.phi1 >= 0 && r.phi2 >= 0) {
    if (phitab2)  // (A/sqrt2)[phi1(x1-t) phi2(x2-t) + phi1(x2-t) phi2(x1-t)]: phitab2 = phi1, phitab = phi2
      c0 = (C * M_SQRT1_2) * (phitab2[r.phi1] * phitab[r.phi2] + phitab2[r.phi2] * phitab[r.phi1]);
    else
      c0 = phitab[r.phi1] * phitab[r.phi2];
  }
  const cd v = c0 - (0.5 * sqrt(gamma)) * sum;
  out[q] = make_double2(v.re, v.im);
}

cudaError_t launch_chi(const ChiRec* recs, int64_t count, const double2* probe_val, const cd* phitab, const cd* etab,
                       const cd* phitab2, const cd* etab2, double C, double gamma, bool incident, double2* out,
                       cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_chi<<<(unsigned)((count + 127) / 128), 128, 0, s>>>(recs, count, probe_val, phitab, etab, phitab2, etab2, C,
                                                        gamma, incident ? 1 : 0, out);
  return cudaGetLastError();
}

cudaError_t launch_measures(const cd* snaps, int64_t nx, int tstep, int64_t nsnap, const cd* e1tab, const cd* e0tab,
                            const cd* phitab, const double* norms, int D, double delta, double gamma, double alpha,
                            double* out, cudaStream_t s) {
  if (nsnap <= 0) return cudaSuccess;
  k_measures<<<(unsigned)nsnap, kMeasThreads, 0, s>>>(snaps, nx, tstep, e1tab, e0tab, phitab, norms, D, delta, gamma,
                                                      alpha, out);
  return cudaGetLastError();
}

}  // namespace fdtd

// N_geo (App. D): the integral of d|det M_t|/dt over the times where it is
// positive, on samples of det M_t: the sum of the increases of |det M| between
// consecutive samples.  Host code.
extern "C" fdtd_status fdtd_geometric_measure(const double* det_m, int64_t n, double* out) {
  if (!out || n < 0 || (n > 0 && !det_m)) return FDTD_ERR_INVALID_ARG;
  double s = 0.0;
  for (int64_t i = 1; i < n; ++i) {
    const double d = fabs(det_m[i]) - fabs(det_m[i - 1]);
    if (d > 0.0) s += d;
  }
  *out = s;
  return FDTD_OK;
}
