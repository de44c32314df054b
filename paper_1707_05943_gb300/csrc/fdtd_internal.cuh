// fdtd_internal.cuh -- types shared by the CUDA translation units of libfdtd.
// Device complex arithmetic, the plan structure and the kernel entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "fdtd.h"

namespace fdtd {

// ---------------------------------------------------------------- complex FP64
struct cd {
  double re, im;
};
__host__ __device__ __forceinline__ cd mk(double r, double i) { return cd{r, i}; }
__host__ __device__ __forceinline__ cd operator+(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ cd operator-(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cd operator-(cd a) { return cd{-a.re, -a.im}; }
__host__ __device__ __forceinline__ cd operator*(cd a, cd b) {
  return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ cd operator*(double s, cd a) { return cd{s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ cd operator*(cd a, double s) { return cd{s * a.re, s * a.im}; }
// acc + a*b with fused multiply-adds
__host__ __device__ __forceinline__ cd cfma(cd a, cd b, cd acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
__host__ __device__ __forceinline__ double cabs2(cd a) { return a.re * a.re + a.im * a.im; }

// ---------------------------------------------------------------- constants
constexpr int kMarchThreads = 512;   // threads per CTA of the FP64 march
constexpr int kMarchP = 8;           // leading columns of a thread's segment kept in registers
constexpr int kMaxTrunc = 64;        // cap on scan / halo truncation depth
constexpr int kMaxGrid = 1024;       // cap on CTAs of the persistent march

// sync words at the start of the workspace
struct SyncWords {
  unsigned int bar_count;
  unsigned int bar_gen;
  unsigned int status;     // fdtd_status latched by the device (0 = ok)
  unsigned int pad;
  long long where;         // row at which a device error was latched
};

// ---------------------------------------------------------------- march args
struct MarchArgs {
  cd* ring;              // R rows x stride
  int64_t stride;        // columns per ring row (>= nx)
  int R;                 // ring rows = D + 2
  const cd* etab;        // e(r delta), r < nt
  const cd* phitab;      // phi(-a - j delta), j < nphi
  const cd* rowscal;     // per row: R1(n), R2(n)  (2 per row)
  const cd* detab;       // E(i-D) - E(i), i < nt + D
  double* norms;         // nt
  double* partials;      // 2 x grid
  cd* snaps;             // nsnap x nx or null
  const int64_t* colsplit;  // grid+1 column starts
  SyncWords* sync;
  int64_t n_begin, n_end;   // rows marched by this launch
  int64_t nx, nt, nphi;
  int D;
  int tstep;
  cd c1, c2, c3;         // update coefficients
  cd gs;                 // -(Gamma/4) / A: mirror-bar source coefficient
  double C;              // psi(x<=-a) prefactor
  double delta;
  int kfix;              // columns that receive a carry (|c2|^kfix < 2^-60)
  int khalo;             // halo columns recomputed left of each CTA range
  int hreuse;            // 1: delay pair sums of the previous row kept in shared memory
  int mid_weight;        // cost of a column of -a < x <= 3a in bulk columns
  cd c2pow[kMaxTrunc + 1];  // c2^0 .. c2^kMaxTrunc
  long long spin_cycles; // bounded wait of the grid barrier
};

// ---------------------------------------------------------------- boundary args
struct BoundaryArgs {
  cd* etab;
  cd* phitab;
  cd* rowscal;
  cd* detab;             // nt + D entries, see k_detab
  double* norms;         // norms[0] is set here (row 0 is the initial condition)
  int64_t nt, nphi;
  int D;
  int init_cond;
  double delta, gamma, omega0, k, alpha, sigma, center;
  double C;
  cd cs;                 // 1/A
  unsigned int* status;  // latched FDTD_ERR_NOT_CONVERGED
};

}  // namespace fdtd

// the plan (opaque to users)
struct fdtd_plan_s {
  fdtd_params p;
  cudaStream_t stream;
  int device;
  int num_sms;
  int grid;              // CTAs of the persistent march
  // derived
  fdtd::cd c1, c2, c3, cs, gs;
  double C;
  // workspace layout (byte offsets)
  size_t ws_need;
  char* ws;
  size_t off_sync, off_etab, off_phi, off_rowscal, off_detab, off_norms, off_hscr, off_partials, off_colsplit, off_ring, off_snaps;
  int64_t stride, nphi, nsnap;
  int R;
  size_t elem;
  int64_t rows_done;     // rows available (0 before set_boundary)
  int state;             // 0 planned, 1 bound, 2 boundary set
  int kfix, khalo;
  size_t march_smem;     // dynamic shared memory of the march (delay pair sums)
  int mid_weight;        // column split weight of -a < x <= 3a
  bool record_errors = true;  // false: keep no message (no host allocation on error paths)
  std::string last_error;
};

// fills a plan without allocating it (fdtd_plan = new + this)
fdtd_status fdtd_plan_fill(fdtd_plan_s* P, const fdtd_params* pin, int32_t n_instances, void* cuda_stream,
                           size_t* workspace_bytes);

namespace fdtd {
// launchers (return cudaError_t)
cudaError_t launch_boundary(const BoundaryArgs& a, cd* hscratch, bool compute_etable, cudaStream_t s);
cudaError_t launch_gamma_star(const int32_t* n, const double* z, double* out, int64_t count, cudaStream_t s);
cudaError_t launch_march_f64(const MarchArgs& a, int grid, size_t smem, cudaStream_t s);
int march_f64_max_grid(int device);
}  // namespace fdtd
