// fdtd_internal.cuh -- types shared by the CUDA translation units of libfdtd.
// Device complex arithmetic, the plan structure and the kernel entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

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

// complex64 compensated march (march_f32c.cu)
constexpr int kF32Threads = 256;     // threads per CTA
constexpr int kF32Band = 256;        // rows per band of the complex64 sweep
constexpr int kGangMax = 64;         // band streams of one complex64 instance at most

// double-float march (march_dw.cu)
constexpr int kDwThreads = 256;      // threads per CTA; two CTAs per SM
constexpr int kDwCtasPerSm = 2;
constexpr int kDwP = 4;              // leading columns of a segment kept in registers
// row pipeline of the FP64 and double-float marches
constexpr int kRowSlack = 32;        // ring rows beyond D+2: how far a CTA may run ahead of its readers
constexpr int kMaxDeps = 4096;       // (cta, lag) entries of the dependency lists, all CTAs together

// sync words at the start of the workspace
struct SyncWords {
  unsigned int bar_count;
  unsigned int bar_gen;
  unsigned int status;     // fdtd_status latched by the device (0 = ok)
  unsigned int pad;
  long long where;         // row at which a device error was latched
};

// ---------------------------------------------------------------- row pipeline
// The persistent marches separate rows without a grid barrier: CTA b publishes
// done[b] = rows it has completed (a release store after its row's stores);
// before row n it waits (acquire loads, bounded) until each CTA it reads has
// completed row n - lag (dep: the smallest lag at which b reads that CTA), and
// until each CTA that reads b has completed row n - 1 - slack (the ring holds
// D + 2 + slack rows, so the slot of row n is free).  Every wait is for a
// strictly earlier row, so no set of waits can close a cycle.
struct RowDeps {
  const int* dep_off;        // grid+1: CTA b's dependencies are dep[dep_off[b] .. dep_off[b+1])
  const int2* dep;           // (cta, lag)
  const int* rd_off;         // grid+1: CTA b's readers are rd[rd_off[b] .. rd_off[b+1])
  const int* rd;
  unsigned long long* done;  // per CTA: rows completed (absolute row index + 1)
};

#ifdef __CUDACC__
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;\n" ::"l"(p), "l"(v) : "memory");
}
// wait until done[cta] > row (rows before n_begin are complete: earlier launches
// finished); false on timeout or when another CTA has latched an error
__device__ __forceinline__ bool wait_row_done(const RowDeps& P, SyncWords* sync, long long spin_cycles,
                                              int64_t n_begin, int cta, int64_t row) {
  if (row < n_begin) return true;
  const unsigned long long need = (unsigned long long)(row + 1);
  if (ld_acquire_u64(&P.done[cta]) >= need) return true;
  const long long t0 = clock64();
  int k = 0;
  for (;;) {
    __nanosleep(64);
    if (ld_acquire_u64(&P.done[cta]) >= need) return true;
    if ((++k & 15) == 0 && *(volatile unsigned int*)&sync->status != 0u) return false;
    if (clock64() - t0 > spin_cycles) return false;
  }
}
// warp 0 of CTA `cta` before row n: returns false (to every lane) if a wait gave up,
// after latching FDTD_ERR_TIMEOUT; the caller's CTA barrier then publishes the result
__device__ __forceinline__ bool row_wait_warp(const RowDeps& P, SyncWords* sync, long long spin_cycles,
                                              int64_t n_begin, int cta, int64_t n, int slack) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int k = P.dep_off[cta] + lane; k < P.dep_off[cta + 1]; k += 32) {
    const int2 d = P.dep[k];
    if (!wait_row_done(P, sync, spin_cycles, n_begin, d.x, n - d.y)) ok = false;
  }
  for (int k = P.rd_off[cta] + lane; k < P.rd_off[cta + 1]; k += 32)
    if (!wait_row_done(P, sync, spin_cycles, n_begin, P.rd[k], n - 1 - slack)) ok = false;
  ok = __all_sync(0xffffffffu, ok);
  __threadfence();  // the rows waited for are visible to every thread after the caller's barrier
  if (!ok && lane == 0 && atomicCAS(&sync->status, 0u, (unsigned)FDTD_ERR_TIMEOUT) == 0u) sync->where = n;
  return ok;
}
#endif

// ---------------------------------------------------------------- march args
struct MarchArgs {
  cd* ring;              // R rows x stride
  int64_t stride;        // columns per ring row (>= nx)
  int R;                 // ring rows = D + 2 + kRowSlack
  const cd* etab;        // e(r delta), r < nt
  const cd* phitab;      // phi(-a - j delta), j < nphi
  const cd* rowscal;     // per row: R1(n), R2(n)  (2 per row)
  const cd* detab;       // E(i-D) - E(i), i < nt + D
  // two different photons (FDTD_IC_TWO_PHOTON_PAIR): psi(x<=-a) = C (phi e + phi2 e2),
  // the bulk sources gain R1'(n) dE2 + R2'(n) phi2; null otherwise
  const cd* phitab2;
  const cd* etab2;
  const cd* rowscal2;
  const cd* detab2;
  double* norms;         // nt
  double* partials;      // (n - n_begin) * grid + cta: the CTA's trapezoid sum of |psi|^2 on row n
  cd* snaps;             // nsnap x nx or null
  const int64_t* colsplit;  // grid+1 column starts
  RowDeps deps;          // row pipeline
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
  long long spin_cycles; // bound of every wait on another CTA
  // probes: points of row n are probe_col[probe_off[n] .. probe_off[n+1]) (null: none);
  // the value of column probe_col[k] goes to probe_val[probe_idx[k]]
  const int* probe_off;
  const int* probe_col;
  const int* probe_idx;
  double2* probe_val;
};

// ---------------------------------------------------------------- double-float march args
// A complex value in double-float: (rh + rl) + i (ih + il), stored as float4
// (rh, ih, rl, il); |rl| <= ulp(rh)/2 once normalised.
struct DwArgs {
  float4* ring;          // R rows x stride, R = D + 2 + kRowSlack
  int64_t stride;
  int R;
  const float4* etabC;   // C e(r delta), r < nt
  const float4* phitab;  // phi(-a - j delta), j < nphi
  const float4* rowscal; // R1(n), R2(n)
  const float4* detab;   // E(i-D) - E(i), i < nt + D
  const float4* etabC2;  // second term of a photon pair (as in MarchArgs), null otherwise
  const float4* phitab2;
  const float4* rowscal2;
  const float4* detab2;
  double* partials;      // (n - n_begin) * grid + cta: sum over the CTA's columns of w_j |psi|^2
  double2* snaps;        // complex128 snapshots or null
  const int64_t* colsplit;
  RowDeps deps;          // row pipeline
  SyncWords* sync;
  int64_t n_begin, n_end;
  int64_t nx, nt, nphi;
  int D, tstep, kfix, khalo, hreuse, mid_weight;
  float4 d1, c2, c3, gs;  // c1 - 1, c2, c3, -(Gamma/4)/A in double-float
  float4 c2pow[kMaxTrunc + 1];
  long long spin_cycles;
  const int* probe_off;  // as in MarchArgs
  const int* probe_col;
  const int* probe_idx;
  double2* probe_val;
};

// ---------------------------------------------------------------- boundary args
struct BoundaryArgs {
  cd* etab;
  cd* phitab;
  cd* rowscal;
  cd* detab;             // nt + D entries, see k_detab
  // FDTD_IC_TWO_PHOTON_PAIR: the second term's tables (null otherwise) and photon
  cd* etab2;
  cd* phitab2;
  cd* rowscal2;
  cd* detab2;
  double k2, alpha2;
  double* norms;         // norms[0] is set here (row 0 is the initial condition)
  int64_t nt, nphi;
  int D;
  int init_cond;
  double delta, gamma, omega0, k, alpha, sigma, center;
  double C;
  cd cs;                 // 1/A
  unsigned int* status;  // latched FDTD_ERR_NOT_CONVERGED
};

// one instance of a complex64 (batched) march, as the device reads it
struct InstDesc {
  int64_t nx, nt, stride, nphi;
  int64_t range[2];        // rows [range[0], range[1]) marched by the current launch; range[1] = rows done
  int D, R, tstep, pad0;
  long long spin;          // clock cycles a bounded wait spins before latching FDTD_ERR_TIMEOUT
  float2 d1, c2, c3, gs;   // c1 - 1, c2, c3, -(Gamma/4)/A
  float2 d1lo, c2lo, c3lo; // their FP32 rounding errors: d1 = d1 + d1lo to ~2^-48 (a coefficient
                           // error is the same at every step, so it would grow linearly along
                           // a characteristic)
  float2 pad1;
  double C, delta;
  float2* ring;            // inner columns j < D: R rows x stride complex64, row-major
  float2* skew;            // columns j >= D: element (n, j) at skew[((n + j - D) mod rd) R + n mod R]
                           // (a warp's 32 rows at one sweep step are 32 consecutive entries)
  int64_t rd;              // nx - D
  float2* snaps;           // or null
  float2* lo_in;           // 2 x dpad: TwoSum remainders of the inner columns (j < D), by row parity
  float2* lo_row;          // nx: remainders of columns j >= D of the last row of the latest band
  float2* lo_edge;         // nt: remainder of column D-1 of every row
  int64_t dpad;            // >= D, a multiple of 8 elements
  unsigned long long* bsync;  // [0] rows whose inner columns are complete; [1 + r] progress of
                              // band stream r: (first row of its band << 32) + columns of the
                              // band's last row done
  double* norms;           // nt
  const cd* etab;          // FP64 tables
  const cd* phitab;
  const float2* etab32;    // FP32 copies
  const float2* phitab32;  // zero-padded: [-(nx - D) - D - 64, 0) and 64 entries past the end
  const float2* detab32;   // zero-padded: [-(nx - D) - 64, 0) and 64 entries past the end
  const float2* rowscal32;
  const float2* bnd32;     // 2 per row: psi(-a, n delta) as FP32 hi and lo
  const double* bnorm;     // per row: (1/2)|psi(-a, n delta)|^2
};

// one entry of the batched march's queue: band stream `stream` of `g` of one instance
struct WorkItem {
  int inst;
  int stream;
  int g;
  int pad;
};

}  // namespace fdtd

// host mirror of one instance of a batched complex64 plan
struct fdtd_batch_inst {
  fdtd_params p;
  size_t off_etab, off_phi, off_rowscal, off_detab, off_norms, off_hscr, off_etab32, off_phi32, off_rowscal32,
      off_detab32, off_ring, off_skew, off_snaps, off_lo, off_bsync, off_bnd, off_bnorm;
  int64_t stride, nphi, nsnap;
  int64_t dpad, nxpad, lo_elems;  // remainders: lo_in 2 x dpad, lo_row nxpad, lo_edge nt
  int64_t padl_e, padl_f;         // zero entries before the FP32 detab and phi tables
  int R, g;                       // ring rows; CTAs that march the instance together
  fdtd::cd c1, c2, c3, cs, gs;
  double C;
  int64_t rows_done;
};

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
  // FDTD_F64_DW plans
  bool dw = false;
  size_t off_dwtab = 0, off_done = 0, off_deps = 0, off_rowout = 0;
  // stimulated-emission plans: one-excitation e0 table and the App. D measures
  size_t off_e0tab = 0, off_meas = 0;
  // photon pairs (FDTD_IC_TWO_PHOTON_PAIR): the second term's tables (0: none)
  size_t off_pair = 0;
  // probes (fdtd_set_probes) and chi points (fdtd_set_chi_points)
  size_t off_probes = 0, off_chi = 0;
  int64_t n_probes = 0, n_chi = 0;
  int64_t rows_per_launch = 0;
  // complex64 (batched) plans
  bool batched = false;
  std::vector<fdtd_batch_inst> inst;
  size_t off_desc = 0, off_order = 0, off_queue = 0, off_eargs = 0, off_stage = 0;
  int nitems = 0;
  int gang_max = 0;          // band streams of one instance at most
  // fdtd_march_graph: the recorded launch sequence of one march length
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_rows = -1;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::string last_error;
  ~fdtd_plan_s() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

// checkpoint / resume (state.cu)
int64_t state_bytes(fdtd_plan_s* P, int inst);
fdtd_status state_readout(fdtd_plan_s* P, int inst, void* dst, int64_t dst_bytes, cudaStream_t s);
fdtd_status state_restore(fdtd_plan_s* P, const void* blob, int64_t nbytes, cudaStream_t s, int64_t* rows_restored);

// fills a plan without allocating it (fdtd_plan = new + this)
fdtd_status fdtd_plan_fill(fdtd_plan_s* P, const fdtd_params* pin, int32_t n_instances, void* cuda_stream,
                           size_t* workspace_bytes);
// complex64 (batched) plans: batch_api.cu
fdtd_status batch_plan_fill(fdtd_plan_s* P, const fdtd_params* pin, int32_t n, void* cuda_stream,
                            size_t* workspace_bytes);
fdtd_status batch_set_boundary(fdtd_plan_s* P, int32_t source, const void* table, int64_t n);
fdtd_status batch_march(fdtd_plan_s* P, int64_t rows);
fdtd_status batch_march_graph(fdtd_plan_s* P, int64_t rows);
int64_t batch_readout_bytes(fdtd_plan_s* P, int32_t inst, int32_t kind);
fdtd_status batch_readout(fdtd_plan_s* P, int32_t inst, int32_t kind, void* dst, int64_t dst_bytes);

namespace fdtd {
// launchers (return cudaError_t)
cudaError_t launch_boundary(const BoundaryArgs& a, cd* hscratch, bool compute_etable, cudaStream_t s);
// the boundary of a photon pair (FDTD_IC_TWO_PHOTON_PAIR): both terms' tables
cudaError_t launch_boundary_pair(const BoundaryArgs& a, cd* hscratch, cd* hscratch2, bool compute_etable,
                                 cudaStream_t s);
// the same work in three steps, so that a batch computes every e-table in one launch
struct EtabArgs {
  BoundaryArgs b;
  cd* h;  // scratch for h(r delta) (two-photon classes)
  int panels;
};
EtabArgs etable_args(const BoundaryArgs& a, cd* hscratch);
cudaError_t launch_boundary_pre(const BoundaryArgs& a, cudaStream_t s);
cudaError_t launch_etable_batch(const EtabArgs* dev_args, int n, int64_t max_nt, cudaStream_t s);
cudaError_t launch_boundary_post(const BoundaryArgs& a, cudaStream_t s);
cudaError_t launch_gamma_star(const int32_t* n, const double* z, double* out, int64_t count, cudaStream_t s);
cudaError_t launch_etable_e0(const BoundaryArgs& a, cd* e0tab, cd* hscratch, cudaStream_t s);
// one point of the two-photon wavefunction chi (Eq. 2), resolved on the host:
// chi = chi0 - (sqrt(Gamma)/2) sum_t w[t] psi_t, psi_t a probe value (kind 1) or
// the exact C phi e of x <= -a (kind 2, phitab[idx] etab[row])
struct ChiRec {
  double w[4];
  int32_t kind[4], idx[4], row[4];
  int32_t phi1, phi2;  // phitab indices of the incident chi0 = phi(x1-t) phi(x2-t); -1: zero
  int32_t pad[2];
};
cudaError_t launch_chi(const ChiRec* recs, int64_t count, const double2* probe_val, const cd* phitab,
                       const cd* etab, const cd* phitab2, const cd* etab2, double C, double gamma, bool incident,
                       double2* out, cudaStream_t s);
cudaError_t launch_measures(const cd* snaps, int64_t nx, int tstep, int64_t nsnap, const cd* e1tab, const cd* e0tab,
                            const cd* phitab, const double* norms, int D, double delta, double gamma, double alpha,
                            double* out, cudaStream_t s);
cudaError_t launch_march_f64(const MarchArgs& a, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_tables32(const InstDesc& I, const cd* detab, const cd* rowscal, cudaStream_t s);
cudaError_t launch_advance(InstDesc* insts, int ninst, int64_t rows, cudaStream_t s);
// where row r of a complex64 instance lives (inner ring and anti-diagonal ring)
struct RowMap {
  float2* ring;
  int64_t stride;
  float2* skew;
  int64_t rd, nx;
  int R, D;
};
// row r between the rings and a row-major buffer: dir 0 gathers into buf, 1 scatters
// buf into the rings, 2 writes zeros into the rings
cudaError_t launch_row_move(const RowMap& m, int64_t r, float2* buf, int dir, cudaStream_t s);
int march_f32c_blocks_per_sm();
}  // namespace fdtd
fdtd::RowMap row_map(fdtd_plan_s* P, int i);  // instance i of a complex64 plan (batch_api.cu)
namespace fdtd {
cudaError_t launch_march_f32c(const InstDesc* insts, const WorkItem* items, int nitems, unsigned int* queue,
                              SyncWords* sync, int grid, cudaStream_t s);
int march_f64_max_grid(int device);
int march_dw_max_grid(int device);
cudaError_t launch_tables_dw(const cd* etab, const cd* phitab, const cd* rowscal, const cd* detab, double C,
                             int64_t nt, int64_t nphi, int D, float4* etabC, float4* phitab_dw, float4* rowscal_dw,
                             float4* detab_dw, cudaStream_t s);
cudaError_t launch_march_dw(const DwArgs& a, int grid, size_t smem, cudaStream_t s);
int march_dw_blocks_per_sm(size_t smem);
cudaError_t launch_norms_rows(const double* partials, int grid, int64_t n_begin, int64_t n_end, const cd* etab,
                             const cd* phitab, const cd* etab2, const cd* phitab2, double C, double delta,
                             double* norms, cudaStream_t s);
cudaError_t launch_row_dw(const float4* src, int64_t nx, double2* dst, cudaStream_t s);
}  // namespace fdtd
