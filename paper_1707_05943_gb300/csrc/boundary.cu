// boundary.cu -- FP64 kernels that build the boundary of the march:
//   * G(n,z) = Gamma(n) gamma*(n,z), the incomplete Gamma function for integer
//     n >= 1 and complex z (App. C);
//   * e(t), the one-excitation atom amplitude that fixes psi(x<=-a,t)
//     (Sec. 2 (b), (c)), one thread per row;
//   * the wavepacket table phi(-a - j delta) and the per-row source scalars.
//
// e(t) for the two-photon classes is built as e(t) = h(t) - h(t-2a) with
//   h(tau) = sum_j (Gamma/2)^j F_j(tau - 2ja),
//   F_j(u) = int_0^u (u-v)^j e^{-W(u-v)} / j!  g(v) dv,  g(v) = sqrt(Gamma/2) phi(-a-v),
// the response of the one-excitation delay equation to the drive
// sqrt(Gamma/2)[phi(-a-t) - phi(a-t)].  For the exponential wavepacket of
// Sec. 2 (b) the integral is closed: F_j(u) = g0 u^{j+1} e^{-kappa u} G(j+1,-ipu)/j!
// with kappa = ik + alpha Gamma/2 and p = k - w0 + i Gamma (1-alpha)/2, which is
// how gamma(n,z) enters (the paper's Sec. 2 (c) series is the same sum
// regrouped).  For the Gaussian wavepacket F_j is integrated by composite
// Gauss-Legendre over the part of [0,u] where the pulse is above e^-40.
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>

#include "fdtd_internal.cuh"

namespace fdtd {

// Gauss-Legendre rule for the Gaussian drive: nodes/weights on [-1,1].
constexpr int kGL = 16;
__constant__ double c_gl_x[kGL];
__constant__ double c_gl_w[kGL];

__device__ __forceinline__ cd cexp_d(cd z) {
  double s, c;
  sincos(z.im, &s, &c);
  double m = exp(z.re);
  return cd{m * c, m * s};
}

// Gamma(n) gamma*(n,z) for integer n >= 1.
//   |z| < n+1 : e^-z sum_i z^i / (n (n+1) ... (n+i))   (terms shrink by |z|/(n+i+1))
//   otherwise : Gamma(n)/z^n - e^-z sum_{i<n} (n-1)!/(n-1-i)! z^-(i+1),
//               the integer-n closed form, whose terms shrink by (n-1-i)/|z|.
__device__ cd gstar_scaled(int n, cd z, unsigned int* status) {
  double az = hypot(z.re, z.im);
  if (az < n + 1.0) {
    cd t = cd{1.0 / n, 0.0}, s = t;
    for (int i = 1; i < 20000; ++i) {
      t = (1.0 / (n + i)) * (t * z);
      s = s + t;
      if (cabs2(t) <= 1e-34 * cabs2(s)) return cexp_d(-z) * s;
    }
    if (status) atomicCAS(status, 0u, (unsigned)FDTD_ERR_NOT_CONVERGED);
    return cexp_d(-z) * s;
  }
  // 1/z
  double d = z.re * z.re + z.im * z.im;
  cd iz = cd{z.re / d, -z.im / d};
  cd lead = iz;
  for (int k = 1; k < n; ++k) lead = (double)k * (lead * iz);
  cd t = iz, s = iz;
  for (int i = 1; i <= n - 1; ++i) {
    t = (double)(n - i) * (t * iz);
    s = s + t;
  }
  return lead - cexp_d(-z) * s;
}

__global__ void k_gamma_star(const int32_t* __restrict__ n, const double* __restrict__ z, double* __restrict__ out,
                             int64_t count) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  cd g = gstar_scaled(n[i], cd{z[2 * i], z[2 * i + 1]}, nullptr);
  out[2 * i] = g.re;
  out[2 * i + 1] = g.im;
}

// phi(x) for x = -(D/2 + j) delta (j >= 0), the incident wavepacket at and left of x = -a.
__device__ cd phi_left(const BoundaryArgs& A, double x) {
  double a = 0.5 * A.D * A.delta;
  if (A.init_cond == FDTD_IC_TWO_PHOTON_GAUSS) {
    double s2 = A.sigma * A.sigma;
    double amp = pow(2.0 * M_PI * s2, -0.25) * exp(-(x - A.center) * (x - A.center) / (4.0 * s2));
    double sn, cs;
    sincos(A.k * x, &sn, &cs);
    return cd{amp * cs, amp * sn};
  }
  if (A.init_cond == FDTD_IC_PLANE_WAVE) {  // Sec. 2 (a): e^{ikx}, A = 1
    double sn, cs;
    sincos(A.k * x, &sn, &cs);
    return cd{cs, sn};
  }
  double ag = A.alpha * A.gamma;
  cd e = cexp_d(cd{0.5 * ag * (x + a), A.k * x});
  double r = sqrt(ag);
  return cd{-r * e.im, r * e.re};  // i sqrt(ag) e
}

// e1(t), Sec. 2 (b): sum_n exp(n log(Gamma u/2) - log n! - W u), u = t - 2na >= 0.
__device__ cd e1_at(const BoundaryArgs& A, double t) {
  double twoa = A.D * A.delta;
  cd W = cd{0.5 * A.gamma, A.omega0};
  cd s = cexp_d(-t * W);
  for (int n = 1;; ++n) {
    double u = t - n * twoa;
    if (u <= 0.0) break;
    double lw = n * log(0.5 * A.gamma * u) - lgamma(n + 1.0);
    s = s + cexp_d(cd{lw - W.re * u, -W.im * u});
  }
  return s;
}

// h(tau) for the exponential wavepacket: sum_j (Gamma/2)^j g0 u^{j+1} e^{-kappa u} G(j+1,-ipu)/j!.
// The plane wave of Sec. 2 (a) is the same sum with alpha = 0 and the packet's
// amplitude i sqrt(alpha Gamma) replaced by 1: g0 = sqrt(Gamma/2) e^{-ika},
// kappa = ik, p = k - w0 + i Gamma/2.
__device__ cd h_exp(const BoundaryArgs& A, double tau, unsigned int* status) {
  if (tau <= 0.0) return cd{0.0, 0.0};
  const bool plane = (A.init_cond == FDTD_IC_PLANE_WAVE);
  const double twoa = A.D * A.delta, a = 0.5 * twoa;
  const double alpha = plane ? 0.0 : A.alpha;
  const double ag = alpha * A.gamma;
  const double kr = 0.5 * ag, ki = A.k;                            // kappa
  const cd mip = cd{0.5 * A.gamma * (1.0 - alpha), -(A.k - A.omega0)};  // -i p
  const double lg2 = log(0.5 * A.gamma);
  // |g0| = sqrt(alpha Gamma^2 / 2) for the packet, sqrt(Gamma / 2) for the plane wave
  const double lg0 = plane ? 0.5 * log(0.5 * A.gamma) : 0.5 * log(0.5 * ag * A.gamma);
  cd s = cd{0.0, 0.0};
  for (int j = 0;; ++j) {
    double u = tau - j * twoa;
    if (u <= 0.0) break;
    double lu = log(u);
    double lw = j * lg2 + (j + 1) * lu - lgamma(j + 1.0) - kr * u;
    // |G(j+1,z)| <= e^{max(0,-Re z)} / (j+1): skip terms below 1e-18 of unit size
    double bound = lw + lg0 + fmax(0.0, -mip.re * u) - log(j + 1.0);
    if (bound < -41.5) continue;
    cd G = gstar_scaled(j + 1, u * mip, status);
    s = s + cexp_d(cd{lw, -ki * u}) * G;
  }
  // g0 = i sqrt(alpha Gamma^2/2) e^{-ika} (packet), sqrt(Gamma/2) e^{-ika} (plane wave)
  cd g0 = cexp_d(cd{lg0, -A.k * a});
  if (!plane) g0 = cd{-g0.im, g0.re};
  return g0 * s;
}

// h(tau) for the Gaussian wavepacket: F_j by composite Gauss-Legendre.
__device__ cd h_gauss(const BoundaryArgs& A, double tau, int panels) {
  if (tau <= 0.0) return cd{0.0, 0.0};
  const double twoa = A.D * A.delta, a = 0.5 * twoa;
  const double s2 = A.sigma * A.sigma;
  const double s0 = -a - A.center;           // the drive peaks at v = s0
  const double half = sqrt(160.0) * A.sigma; // (v-s0)^2/(4 s2) <= 40 inside
  const double lg2 = log(0.5 * A.gamma);
  const double lnorm = 0.5 * log(0.5 * A.gamma) - 0.25 * log(2.0 * M_PI * s2);
  const double Wr = 0.5 * A.gamma, Wi = A.omega0;
  cd tot = cd{0.0, 0.0};
  for (int j = 0;; ++j) {
    double u = tau - j * twoa;
    if (u <= 0.0) break;
    double lo = fmax(0.0, s0 - half), hi = fmin(u, s0 + half);
    if (hi <= lo) continue;
    // bound of (Gamma/2)^j (u-v)^j e^{-Gamma(u-v)/2} / j! over v in [lo,hi]
    double lgj = lgamma(j + 1.0);
    double smin = u - hi, smax = u - lo;
    double sst = fmin(fmax(2.0 * j / A.gamma, smin), smax);
    double lb = j * lg2 - lgj - Wr * sst + (j > 0 ? j * log(fmax(sst, 1e-300)) : 0.0);
    if (lb + lnorm + log(hi - lo + 1e-300) < -41.5) continue;
    cd F = cd{0.0, 0.0};
    double h = (hi - lo) / panels;
    if (Wi == A.k) {
      // resonant carrier: the phase -Wi s + k x = -Wi u - k a is the same at every
      // node, so the quadrature sums a real integrand and takes the phase once
      double Fr = 0.0;
      for (int q = 0; q < panels; ++q) {
        double c0 = lo + (q + 0.5) * h;
        for (int i = 0; i < kGL; ++i) {
          double v = c0 + 0.5 * h * c_gl_x[i];
          double s = u - v;
          if (j > 0 && s <= 0.0) continue;
          double x = -a - v;
          double re = j * lg2 - lgj - Wr * s - (x - A.center) * (x - A.center) / (4.0 * s2) + lnorm;
          if (j > 0) re += j * log(s);
          Fr += (0.5 * h * c_gl_w[i]) * exp(re);
        }
      }
      double sn, cs;
      sincos(-Wi * u - A.k * a, &sn, &cs);
      F = cd{Fr * cs, Fr * sn};
    } else {
      for (int q = 0; q < panels; ++q) {
        double c0 = lo + (q + 0.5) * h;
        for (int i = 0; i < kGL; ++i) {
          double v = c0 + 0.5 * h * c_gl_x[i];
          double s = u - v;
          if (j > 0 && s <= 0.0) continue;
          double x = -a - v;
          double re = j * lg2 - lgj - Wr * s - (x - A.center) * (x - A.center) / (4.0 * s2) + lnorm;
          if (j > 0) re += j * log(s);
          double im = -Wi * s + A.k * x;
          F = F + (0.5 * h * c_gl_w[i]) * cexp_d(cd{re, im});
        }
      }
    }
    tot = tot + F;
  }
  return tot;
}

// pass 1: e(r delta) for stimulated emission, h(r delta) for the two-photon classes
__device__ __forceinline__ void etable_row(const EtabArgs& E, int64_t r) {
  const BoundaryArgs& A = E.b;
  if (r >= A.nt) return;
  double t = r * A.delta;
  if (A.init_cond == FDTD_IC_STIM_EMISSION) {
    A.etab[r] = e1_at(A, t);
  } else if (A.init_cond == FDTD_IC_TWO_PHOTON_EXP || A.init_cond == FDTD_IC_PLANE_WAVE) {
    E.h[r] = h_exp(A, t, A.status);
  } else {
    E.h[r] = h_gauss(A, t, E.panels);
  }
}
__global__ void k_etable_pass1(const EtabArgs E) { etable_row(E, blockIdx.x * (int64_t)blockDim.x + threadIdx.x); }
// every instance of a batch in one launch: blockIdx.y is the instance
__global__ void k_etable_pass1_batch(const EtabArgs* Es) {
  etable_row(Es[blockIdx.y], blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

// pass 2: e(r delta) = h(r delta) - h((r-D) delta)
__device__ __forceinline__ void etable_diff(const EtabArgs& E, int64_t r) {
  const BoundaryArgs& A = E.b;
  if (r >= A.nt || A.init_cond == FDTD_IC_STIM_EMISSION) return;
  cd v = E.h[r];
  if (r >= A.D) v = v - E.h[r - A.D];
  A.etab[r] = v;
}
__global__ void k_etable_pass2(const EtabArgs E) { etable_diff(E, blockIdx.x * (int64_t)blockDim.x + threadIdx.x); }
__global__ void k_etable_pass2_batch(const EtabArgs* Es) {
  etable_diff(Es[blockIdx.y], blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

// phi table and per-row source scalars.
//   phitab[j]   = phi(-(D/2 + j) delta)
//   rowscal[2n] = R1(n) = (1/A)(-Gamma/4) C P(n), the mirror bars of lines 2-3 of
//                 Eq. 1 where both bars lie in x <= -a:
//                 P(n) = phi(-n-D/2) + phi(-n-D/2+1) - phi(-n+D/2) - phi(-n+D/2+1)  (units of delta)
//   rowscal[2n+1] = R2(n) = (1/A) sqrt(Gamma) [phi((-D/2-n+1/2) delta) - phi((D/2-n+1/2) delta)],
//                 the chi term of line 4 for identical photons chi(x1,x2,0) = phi(x1) phi(x2).
__global__ void k_phitab(const BoundaryArgs A) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= A.nphi) return;
  const int Dh = A.D / 2;
  A.phitab[j] = phi_left(A, -(double)(Dh + j) * A.delta);
}

__global__ void k_rowscal(const BoundaryArgs A) {
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= A.nt) return;
  const int D = A.D, Dh = D / 2;
  cd P = A.phitab[n];
  if (n >= 1) P = P + A.phitab[n - 1];
  if (n >= D) P = P - A.phitab[n - D];
  if (n >= D + 1) P = P - A.phitab[n - D - 1];
  cd R1 = (-0.25 * A.gamma * A.C) * (A.cs * P);
  cd R2 = cd{0.0, 0.0};
  if (A.init_cond != FDTD_IC_STIM_EMISSION) {
    cd f1 = (n >= 1) ? phi_left(A, (-Dh - (double)n + 0.5) * A.delta) : cd{0.0, 0.0};
    cd f2 = (n >= D + 1) ? phi_left(A, (Dh - (double)n + 0.5) * A.delta) : cd{0.0, 0.0};
    R2 = sqrt(A.gamma) * (A.cs * (f1 - f2));
  }
  A.rowscal[2 * n] = R1;
  A.rowscal[2 * n + 1] = R2;
}

// dEtab[i] = E(i-D) - E(i), E(r) = theta(r) e(r delta) (theta(0) = 1/2, E = 0 outside
// 0 <= r < nt): the e-dependence of the mirror sources S2 + S3 beyond x > 3a, indexed by
// i = r2 + D with r2 = n - m - D/2.
__global__ void k_detab(const BoundaryArgs A) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= A.nt + A.D) return;
  auto E = [&](int64_t r) -> cd {
    if (r < 0 || r >= A.nt) return cd{0.0, 0.0};
    return (r == 0) ? 0.5 * A.etab[0] : A.etab[r];
  };
  A.detab[i] = E(i - A.D) - E(i);
}

// norms[0] = delta * (1/2) |psi(-a, 0)|^2: psi(x>-a, 0) = 0 in every class.
__global__ void k_norm0(const BoundaryArgs A) {
  cd v = A.phitab[0] * A.etab[0];
  if (A.phitab2) v = v + A.phitab2[0] * A.etab2[0];  // second term of a photon pair
  v = A.C * v;
  A.norms[0] = A.delta * 0.5 * cabs2(v);
}

// Row scalars of a photon pair (Sec. 2 (c)).  psi(x<=-a) = A [phi1(x-t) e0^(2)(t) +
// phi2(x-t) e0^(1)(t)] is stored as C (phitab etab + phitab2 etab2) with phitab = phi2,
// etab = e0^(1), phitab2 = phi1, etab2 = e0^(2), C = A.  The mirror bars then give
// R1(n) dE(i) + R1'(n) dE2(i) with R1 from the phi2 table and R1' from the phi1 table
// (as k_rowscal), and the chi term of line 4 with chi(x1,x2,0) = (A/sqrt2)[phi1(x1)
// phi2(x2) + phi1(x2) phi2(x1)] gives R2(n) phi2(r2) + R2'(n) phi1(r2), with
//   R2(n)  = (1/A_coef) sqrt(Gamma) (A/sqrt2) [phi1(x_c-...) ...] built from phi1,
//   R2'(n) the same from phi2 (A_coef the update's A, entering as cs = 1/A_coef).
__global__ void k_rowscal_pair(const BoundaryArgs A, const BoundaryArgs A1, const BoundaryArgs A2) {
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= A.nt) return;
  const int D = A.D, Dh = D / 2;
  auto P = [&](const cd* tab) {
    cd v = tab[n];
    if (n >= 1) v = v + tab[n - 1];
    if (n >= D) v = v - tab[n - D];
    if (n >= D + 1) v = v - tab[n - D - 1];
    return v;
  };
  const double g = -0.25 * A.gamma * A.C;
  A.rowscal[2 * n] = g * (A.cs * P(A.phitab));
  A.rowscal2[2 * n] = g * (A.cs * P(A.phitab2));
  auto diff = [&](const BoundaryArgs& B) {  // phi_B(t1) - phi_B(t2) at the square centre
    cd f1 = (n >= 1) ? phi_left(B, (-Dh - (double)n + 0.5) * A.delta) : cd{0.0, 0.0};
    cd f2 = (n >= D + 1) ? phi_left(B, (Dh - (double)n + 0.5) * A.delta) : cd{0.0, 0.0};
    return f1 - f2;
  };
  const double h = sqrt(A.gamma) * A.C * M_SQRT1_2;
  A.rowscal[2 * n + 1] = h * (A.cs * diff(A1));   // multiplies phitab = phi2
  A.rowscal2[2 * n + 1] = h * (A.cs * diff(A2));  // multiplies phitab2 = phi1
}

static bool g_gl_ready[64] = {false};

static cudaError_t upload_gl(int dev) {
  if (dev >= 0 && dev < 64 && g_gl_ready[dev]) return cudaSuccess;
  double x[kGL], w[kGL];
  const int N = kGL;
  for (int i = 0; i < N; ++i) {
    double z = cos(M_PI * (i + 0.75) / (N + 0.5)), p0 = 1, p1 = z, dp = 1;
    for (int it = 0; it < 100; ++it) {
      p0 = 1.0;
      p1 = z;
      for (int k = 2; k <= N; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = N * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    p0 = 1.0;
    p1 = z;
    for (int k = 2; k <= N; ++k) {
      double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    dp = N * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  cudaError_t e = cudaMemcpyToSymbol(c_gl_x, x, sizeof x);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_gl_w, w, sizeof w);
  if (e == cudaSuccess && dev >= 0 && dev < 64) g_gl_ready[dev] = true;
  return e;
}

EtabArgs etable_args(const BoundaryArgs& a, cd* hscratch) {
  EtabArgs E;
  E.b = a;
  E.h = hscratch;
  // panels of 16 Gauss-Legendre nodes: 4 over the pulse window (+-12.6 sigma; against a
  // 32-panel sum the rule is already at FP64 rounding, 6e-15 relative, where 2 panels
  // leave 7e-10), plus two per oscillation of e^{i(w0-k)v} across the window
  double win = 2.0 * sqrt(160.0) * a.sigma;
  E.panels = 4 + 2 * (int)ceil(fabs(a.omega0 - a.k) * win / (2.0 * M_PI));
  return E;
}

// tables that do not need e(t): phi table and per-row source scalars
cudaError_t launch_boundary_pre(const BoundaryArgs& a, cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaError_t e = upload_gl(dev);
  if (e != cudaSuccess) return e;
  const int T = 128;
  k_phitab<<<(unsigned)((a.nphi + T - 1) / T), T, 0, s>>>(a);
  k_rowscal<<<(unsigned)((a.nt + T - 1) / T), T, 0, s>>>(a);
  return cudaGetLastError();
}

// e(t) of n instances whose EtabArgs sit in device memory, one launch per pass
cudaError_t launch_etable_batch(const EtabArgs* dev_args, int n, int64_t max_nt, cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaError_t e = upload_gl(dev);
  if (e != cudaSuccess || n <= 0) return e;
  for (int i0 = 0; i0 < n; i0 += 65535) {  // grid.y limit
    const unsigned m = (unsigned)std::min(65535, n - i0);
    k_etable_pass1_batch<<<dim3((unsigned)((max_nt + 63) / 64), m), 64, 0, s>>>(dev_args + i0);
    k_etable_pass2_batch<<<dim3((unsigned)((max_nt + 127) / 128), m), 128, 0, s>>>(dev_args + i0);
  }
  return cudaGetLastError();
}

// tables that need e(t): the initial norm and the mirror-source differences
cudaError_t launch_boundary_post(const BoundaryArgs& a, cudaStream_t s) {
  const int T = 128;
  k_norm0<<<1, 1, 0, s>>>(a);
  k_detab<<<(unsigned)((a.nt + a.D + T - 1) / T), T, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_boundary(const BoundaryArgs& a, cd* hscratch, bool compute_etable, cudaStream_t s) {
  cudaError_t e = launch_boundary_pre(a, s);
  if (e != cudaSuccess) return e;
  if (compute_etable) {
    const int T = 128;
    EtabArgs E = etable_args(a, hscratch);
    k_etable_pass1<<<(unsigned)((a.nt + 63) / 64), 64, 0, s>>>(E);
    if (a.init_cond != FDTD_IC_STIM_EMISSION) k_etable_pass2<<<(unsigned)((a.nt + T - 1) / T), T, 0, s>>>(E);
  }
  return launch_boundary_post(a, s);
}

// e0 of the one-excitation sector for the exponential packet of a stimulated-
// emission plan (the atom starting in its ground state; App. D uses it): the
// two-photon-class e-table passes with the same photon, written to e0tab
cudaError_t launch_etable_e0(const BoundaryArgs& a, cd* e0tab, cd* hscratch, cudaStream_t s) {
  BoundaryArgs b = a;
  b.init_cond = FDTD_IC_TWO_PHOTON_EXP;
  b.etab = e0tab;
  EtabArgs E = etable_args(b, hscratch);
  k_etable_pass1<<<(unsigned)((a.nt + 63) / 64), 64, 0, s>>>(E);
  k_etable_pass2<<<(unsigned)((a.nt + 127) / 128), 128, 0, s>>>(E);
  return cudaGetLastError();
}

cudaError_t launch_boundary_pair(const BoundaryArgs& a, cd* hscratch, cd* hscratch2, bool compute_etable,
                                 cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaError_t e = upload_gl(dev);
  if (e != cudaSuccess) return e;
  // each photon as an exponential packet of its own
  BoundaryArgs A1 = a, A2 = a;
  A1.init_cond = A2.init_cond = FDTD_IC_TWO_PHOTON_EXP;
  A2.k = a.k2;
  A2.alpha = a.alpha2;
  const int T = 128;
  BoundaryArgs t = A2;  // phitab = phi2
  t.phitab = a.phitab;
  k_phitab<<<(unsigned)((a.nphi + T - 1) / T), T, 0, s>>>(t);
  t = A1;  // phitab2 = phi1
  t.phitab = a.phitab2;
  k_phitab<<<(unsigned)((a.nphi + T - 1) / T), T, 0, s>>>(t);
  k_rowscal_pair<<<(unsigned)((a.nt + T - 1) / T), T, 0, s>>>(a, A1, A2);
  if (compute_etable) {
    BoundaryArgs e1 = A1, e2 = A2;  // etab = e0^(1), etab2 = e0^(2)
    e1.etab = a.etab;
    e2.etab = a.etab2;
    EtabArgs E1 = etable_args(e1, hscratch), E2 = etable_args(e2, hscratch2);
    k_etable_pass1<<<(unsigned)((a.nt + 63) / 64), 64, 0, s>>>(E1);
    k_etable_pass1<<<(unsigned)((a.nt + 63) / 64), 64, 0, s>>>(E2);
    k_etable_pass2<<<(unsigned)((a.nt + T - 1) / T), T, 0, s>>>(E1);
    k_etable_pass2<<<(unsigned)((a.nt + T - 1) / T), T, 0, s>>>(E2);
  }
  k_norm0<<<1, 1, 0, s>>>(a);
  k_detab<<<(unsigned)((a.nt + a.D + T - 1) / T), T, 0, s>>>(a);
  BoundaryArgs d2 = a;  // detab2 from etab2
  d2.etab = a.etab2;
  d2.detab = a.detab2;
  k_detab<<<(unsigned)((a.nt + a.D + T - 1) / T), T, 0, s>>>(d2);
  return cudaGetLastError();
}

cudaError_t launch_gamma_star(const int32_t* n, const double* z, double* out, int64_t count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const int T = 128;
  k_gamma_star<<<(unsigned)((count + T - 1) / T), T, 0, s>>>(n, z, out, count);
  return cudaGetLastError();
}

}  // namespace fdtd
