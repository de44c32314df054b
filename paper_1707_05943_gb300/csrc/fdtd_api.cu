// fdtd_api.cu -- host side of the C ABI declared in include/fdtd.h: parameter
// validation and derivation (Table 1, App. A/B), workspace layout, launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "fdtd_internal.cuh"

using fdtd::cd;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

fdtd_status fail(fdtd_plan_t p, fdtd_status s, const char* msg) {
  if (p && p->record_errors) p->last_error = msg;
  return s;
}

fdtd_status cuda_fail(fdtd_plan_t p, cudaError_t e, const char* where) {
  if (p && p->record_errors) {
    p->last_error = where;
    p->last_error += ": ";
    p->last_error += cudaGetErrorString(e);
  }
  return FDTD_ERR_CUDA;
}

cd cdiv(cd a, cd b) {
  double d = b.re * b.re + b.im * b.im;
  return cd{(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
double cabsh(cd a) { return hypot(a.re, a.im); }

// smallest k >= 1 with |x|^k < 2^-60 (x != 0), capped
int trunc_depth(double ax, int cap) {
  if (ax <= 0.0) return 1;
  if (ax >= 1.0) return cap + 1;
  double k = ceil(-60.0 * log(2.0) / log(ax));
  if (k < 1) k = 1;
  return (k > cap) ? cap + 1 : (int)k;
}

template <class T>
T* at(fdtd_plan_t p, size_t off) {
  return reinterpret_cast<T*>(p->ws + off);
}

}  // namespace

extern "C" {

const char* fdtd_status_string(fdtd_status s) {
  switch (s) {
    case FDTD_OK: return "ok";
    case FDTD_ERR_INVALID_ARG: return "invalid argument";
    case FDTD_ERR_UNSUPPORTED: return "unsupported";
    case FDTD_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case FDTD_ERR_CUDA: return "CUDA error";
    case FDTD_ERR_TIMEOUT: return "device-side wait timed out";
    case FDTD_ERR_BOUNDS: return "device-side index out of bounds";
    case FDTD_ERR_NOT_CONVERGED: return "boundary series did not converge";
    case FDTD_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* fdtd_last_error(fdtd_plan_t p) { return p ? p->last_error.c_str() : ""; }

}  // extern "C"

// Validate parameters and fill a caller-provided plan (no device memory is
// touched).  Shared by fdtd_plan and the no-allocation entry point.
fdtd_status fdtd_plan_fill(fdtd_plan_s* P, const fdtd_params* pin, int32_t n_instances, void* cuda_stream,
                           size_t* workspace_bytes) {
  if (pin->struct_size != sizeof(fdtd_params)) return FDTD_ERR_INVALID_ARG;
  if (n_instances != 1) return FDTD_ERR_UNSUPPORTED;
  const fdtd_params& p = *pin;
  if (p.D < 2 || (p.D & 1) || p.nx < p.D || p.nt < 1) return FDTD_ERR_INVALID_ARG;
  if (!(p.delta > 0) || !(p.gamma > 0) || !isfinite(p.omega0) || !isfinite(p.k)) return FDTD_ERR_INVALID_ARG;
  if (p.init_cond < FDTD_IC_STIM_EMISSION || p.init_cond > FDTD_IC_TWO_PHOTON_GAUSS) return FDTD_ERR_INVALID_ARG;
  if (p.init_cond != FDTD_IC_TWO_PHOTON_GAUSS && !(p.alpha > 0)) return FDTD_ERR_INVALID_ARG;
  if (p.init_cond == FDTD_IC_TWO_PHOTON_GAUSS && !(p.sigma > 0)) return FDTD_ERR_INVALID_ARG;
  if (p.tstep < -1 || p.rows_per_launch < 0) return FDTD_ERR_INVALID_ARG;
  if (p.cluster_ctas < 0 || p.cluster_ctas > 8 || p.mid_weight < 0 || p.mid_weight > 4096) return FDTD_ERR_INVALID_ARG;
  if (p.precision != FDTD_F64) return FDTD_ERR_UNSUPPORTED;

  P->p = p;
  P->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&P->device);
  if (e != cudaSuccess) return FDTD_ERR_CUDA;
  cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
  int maxg = fdtd::march_f64_max_grid(P->device);
  if (maxg <= 0) return FDTD_ERR_CUDA;
  // one CTA per SM, but at least 64 columns per CTA
  int grid = P->num_sms < maxg ? P->num_sms : maxg;
  if ((int64_t)grid > (p.nx + 63) / 64) grid = (int)((p.nx + 63) / 64);
  if (grid > fdtd::kMaxGrid) grid = fdtd::kMaxGrid;
  if (grid < 1) grid = 1;
  P->grid = grid;

  // coefficients (Eq. 3a-c applied to line 1 of Eq. 1; App. A)
  const cd W = cd{0.5 * p.gamma, p.omega0};
  const cd A = cd{1.0 / p.delta + W.re / 4.0, W.im / 4.0};
  const cd B = cd{1.0 / p.delta - W.re / 4.0, -W.im / 4.0};
  P->cs = cdiv(cd{1.0, 0.0}, A);
  P->c1 = cdiv(B, A);
  P->c2 = cdiv(cd{-W.re / 4.0, -W.im / 4.0}, A);
  P->c3 = (p.gamma / 8.0) * P->cs;
  P->gs = (-p.gamma / 4.0) * P->cs;
  P->C = (p.init_cond == FDTD_IC_STIM_EMISSION) ? 1.0 : sqrt(2.0);

  const double ac2 = cabsh(P->c2);
  P->kfix = trunc_depth(ac2, fdtd::kMaxTrunc);
  P->khalo = P->kfix;
  if (P->kfix > fdtd::kMaxTrunc)
    return FDTD_ERR_UNSUPPORTED;  // |c2| too close to 1 (delta far too coarse)

  // workspace layout
  P->R = p.D + 2;
  P->elem = sizeof(cd);
  // row pitch: a multiple of 32 columns plus 32, so that ring rows are never a
  // power-of-two number of bytes apart (rows read together would share L2 slices)
  P->stride = (p.nx + 31) / 32 * 32 + 32;
  P->nphi = p.nt + 3 * (int64_t)p.D + 8;
  P->nsnap = (p.tstep >= 0) ? (p.nt - 1) / (p.tstep + 1) + 1 : 0;
  size_t off = 0;
  P->off_sync = off;     off = align_up(off + sizeof(fdtd::SyncWords));
  P->off_etab = off;     off = align_up(off + sizeof(cd) * (size_t)p.nt);
  P->off_phi = off;      off = align_up(off + sizeof(cd) * (size_t)P->nphi);
  P->off_rowscal = off;  off = align_up(off + 2 * sizeof(cd) * (size_t)p.nt);
  P->off_detab = off;    off = align_up(off + sizeof(cd) * (size_t)(p.nt + p.D));
  P->off_norms = off;    off = align_up(off + sizeof(double) * (size_t)p.nt);
  P->off_hscr = off;     off = align_up(off + sizeof(cd) * (size_t)p.nt);
  P->off_partials = off; off = align_up(off + 2 * sizeof(double) * (size_t)grid);
  P->off_colsplit = off; off = align_up(off + sizeof(int64_t) * (size_t)(grid + 1));
  P->off_ring = off;     off = align_up(off + P->elem * (size_t)P->R * (size_t)P->stride);
  P->off_snaps = off;    off = align_up(off + P->elem * (size_t)P->nsnap * (size_t)p.nx);
  P->ws_need = off;
  P->state = 0;
  *workspace_bytes = P->ws_need;
  return FDTD_OK;
}

extern "C" {

fdtd_status fdtd_plan(const fdtd_params* pin, int32_t n_instances, void* cuda_stream, size_t* workspace_bytes,
                      fdtd_plan_t* out) {
  if (!pin || !workspace_bytes || !out) return FDTD_ERR_INVALID_ARG;
  *out = nullptr;
  fdtd_plan_t P = new (std::nothrow) fdtd_plan_s();
  if (!P) return FDTD_ERR_INVALID_ARG;
  fdtd_status st = (pin->struct_size == sizeof(fdtd_params) && pin->precision == FDTD_F32_COMP)
                       ? batch_plan_fill(P, pin, n_instances, cuda_stream, workspace_bytes)
                       : fdtd_plan_fill(P, pin, n_instances, cuda_stream, workspace_bytes);
  if (st != FDTD_OK) {
    delete P;
    return st;
  }
  *out = P;
  return FDTD_OK;
}

fdtd_status fdtd_bind_workspace(fdtd_plan_t P, void* device_ptr, size_t bytes) {
  if (!P) return FDTD_ERR_INVALID_ARG;
  if (!device_ptr || bytes < P->ws_need || (reinterpret_cast<uintptr_t>(device_ptr) % kAlign))
    return fail(P, FDTD_ERR_WORKSPACE, "workspace missing, smaller than fdtd_plan reported, or not 256-byte aligned");
  P->ws = static_cast<char*>(device_ptr);
  P->state = 1;
  P->rows_done = 0;
  return FDTD_OK;
}

fdtd_status fdtd_set_boundary(fdtd_plan_t P, int32_t source, const void* device_table, int64_t n) {
  if (!P) return FDTD_ERR_INVALID_ARG;
  if (P->state < 1) return fail(P, FDTD_ERR_STATE, "fdtd_set_boundary before fdtd_bind_workspace");
  if (P->batched) return batch_set_boundary(P, source, device_table, n);
  const fdtd_params& p = P->p;
  if (source != FDTD_BOUNDARY_ANALYTIC && source != FDTD_BOUNDARY_TABLE)
    return fail(P, FDTD_ERR_INVALID_ARG, "unknown boundary source");
  if (source == FDTD_BOUNDARY_TABLE && (!device_table || n != p.nt))
    return fail(P, FDTD_ERR_INVALID_ARG, "boundary table must hold nt complex128 values");
  cudaStream_t s = P->stream;
  cudaError_t e;
  // zero sync words, ring, norms, snapshots
  e = cudaMemsetAsync(P->ws + P->off_sync, 0, sizeof(fdtd::SyncWords), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->ws + P->off_ring, 0, P->elem * (size_t)P->R * (size_t)P->stride, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->ws + P->off_norms, 0, sizeof(double) * (size_t)p.nt, s);
  if (e == cudaSuccess && P->nsnap)
    e = cudaMemsetAsync(P->ws + P->off_snaps, 0, P->elem * (size_t)P->nsnap * (size_t)p.nx, s);
  if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemsetAsync");
  if (source == FDTD_BOUNDARY_TABLE) {
    e = cudaMemcpyAsync(P->ws + P->off_etab, device_table, sizeof(cd) * (size_t)p.nt, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemcpyAsync(table)");
  }
  // column split: equal cost per CTA, with the region -a < x <= 3a (2D columns,
  // read through the general path) weighted kMidWeight
  // (measured: a column of -a < x <= 3a costs ~16 bulk columns in FP64)
  const int kMidWeight = p.mid_weight > 0 ? p.mid_weight : 16;
  P->mid_weight = kMidWeight;
  int64_t split[fdtd::kMaxGrid + 1];
  {
    const int64_t mid = (2 * (int64_t)p.D < p.nx) ? 2 * (int64_t)p.D : p.nx;
    const double total = (double)kMidWeight * mid + (double)(p.nx - mid);
    split[0] = 0;
    for (int b = 1; b < P->grid; ++b) {
      double target = total * b / P->grid;
      int64_t j = (target <= kMidWeight * mid) ? (int64_t)(target / kMidWeight) : mid + (int64_t)(target - kMidWeight * mid);
      if (j < split[b - 1]) j = split[b - 1];
      if (j > p.nx) j = p.nx;
      split[b] = j;
    }
    split[P->grid] = p.nx;
  }
  {
    // shared memory for the delay pair sums: khalo + the widest CTA range
    int64_t maxL = 0;
    for (int b = 0; b < P->grid; ++b) maxL = (split[b + 1] - split[b] > maxL) ? split[b + 1] - split[b] : maxL;
    size_t need = sizeof(cd) * (size_t)(maxL + P->khalo);
    P->march_smem = (need <= size_t(200) * 1024) ? need : 0;
  }
  e = cudaMemcpyAsync(P->ws + P->off_colsplit, split, sizeof(int64_t) * (size_t)(P->grid + 1), cudaMemcpyHostToDevice,
                      s);
  if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemcpyAsync(colsplit)");
  // a copy from pageable memory is staged before cudaMemcpyAsync returns
  fdtd::BoundaryArgs a;
  a.etab = at<cd>(P, P->off_etab);
  a.phitab = at<cd>(P, P->off_phi);
  a.rowscal = at<cd>(P, P->off_rowscal);
  a.detab = at<cd>(P, P->off_detab);
  a.nt = p.nt;
  a.nphi = P->nphi;
  a.D = p.D;
  a.init_cond = p.init_cond;
  a.delta = p.delta;
  a.gamma = p.gamma;
  a.omega0 = p.omega0;
  a.k = p.k;
  a.alpha = p.alpha;
  a.sigma = p.sigma;
  a.center = p.center;
  a.C = P->C;
  a.cs = P->cs;
  a.status = &at<fdtd::SyncWords>(P, P->off_sync)->status;
  a.norms = at<double>(P, P->off_norms);
  e = fdtd::launch_boundary(a, at<cd>(P, P->off_hscr), source == FDTD_BOUNDARY_ANALYTIC, s);
  if (e != cudaSuccess) return cuda_fail(P, e, "boundary kernels");
  P->rows_done = 1;
  P->state = 2;
  return FDTD_OK;
}

fdtd_status fdtd_march_graph(fdtd_plan_t P, int64_t n_rows) {
  if (!P) return FDTD_ERR_INVALID_ARG;
  if (!P->batched) return fail(P, FDTD_ERR_UNSUPPORTED, "fdtd_march_graph needs an FDTD_F32_COMP plan");
  if (P->state < 2) return fail(P, FDTD_ERR_STATE, "fdtd_march_graph before fdtd_set_boundary");
  if (n_rows < 0) return fail(P, FDTD_ERR_INVALID_ARG, "n_rows < 0");
  return batch_march_graph(P, n_rows);
}

fdtd_status fdtd_march(fdtd_plan_t P, int64_t n_rows) {
  if (!P) return FDTD_ERR_INVALID_ARG;
  if (P->state < 2) return fail(P, FDTD_ERR_STATE, "fdtd_march before fdtd_set_boundary");
  if (n_rows < 0) return fail(P, FDTD_ERR_INVALID_ARG, "n_rows < 0");
  if (P->batched) return batch_march(P, n_rows);
  const fdtd_params& p = P->p;
  int64_t end = P->rows_done + n_rows;
  if (end > p.nt) end = p.nt;
  if (end <= P->rows_done) return FDTD_OK;
  fdtd::MarchArgs a;
  memset(&a, 0, sizeof a);
  a.ring = at<cd>(P, P->off_ring);
  a.stride = P->stride;
  a.R = P->R;
  a.etab = at<cd>(P, P->off_etab);
  a.phitab = at<cd>(P, P->off_phi);
  a.rowscal = at<cd>(P, P->off_rowscal);
  a.detab = at<cd>(P, P->off_detab);
  a.norms = at<double>(P, P->off_norms);
  a.partials = at<double>(P, P->off_partials);
  a.snaps = P->nsnap ? at<cd>(P, P->off_snaps) : nullptr;
  a.colsplit = at<int64_t>(P, P->off_colsplit);
  a.sync = at<fdtd::SyncWords>(P, P->off_sync);
  a.nx = p.nx;
  a.nt = p.nt;
  a.nphi = P->nphi;
  a.D = p.D;
  a.tstep = p.tstep;
  a.c1 = P->c1;
  a.c2 = P->c2;
  a.c3 = P->c3;
  a.gs = P->gs;
  a.C = P->C;
  a.delta = p.delta;
  a.kfix = P->kfix;
  a.khalo = P->khalo;
  a.hreuse = P->march_smem > 0 ? 1 : 0;
  a.mid_weight = P->mid_weight;
  a.c2pow[0] = cd{1.0, 0.0};
  for (int k = 1; k <= fdtd::kMaxTrunc; ++k) a.c2pow[k] = a.c2pow[k - 1] * P->c2;
  a.spin_cycles = 4000000000LL;  // ~2 s at 2 GHz
  const int64_t per = p.rows_per_launch > 0 ? p.rows_per_launch : 4096;
  for (int64_t n0 = P->rows_done; n0 < end; n0 += per) {
    a.n_begin = n0;
    a.n_end = (n0 + per < end) ? n0 + per : end;
    cudaError_t e = fdtd::launch_march_f64(a, P->grid, P->march_smem, P->stream);
    if (e != cudaSuccess) return cuda_fail(P, e, "march launch");
  }
  P->rows_done = end;
  return FDTD_OK;
}

int64_t fdtd_readout_bytes(fdtd_plan_t P, int32_t kind) {
  if (!P) return -1;
  if (P->batched) return batch_readout_bytes(P, 0, kind);
  const fdtd_params& p = P->p;
  switch (kind) {
    case FDTD_READ_ROW: return (int64_t)P->elem * p.nx;
    case FDTD_READ_NORMS: return (int64_t)sizeof(double) * P->rows_done;
    case FDTD_READ_SNAPSHOTS: {
      if (!P->nsnap || P->rows_done == 0) return 0;
      int64_t ns = (P->rows_done - 1) / (p.tstep + 1) + 1;
      return (int64_t)P->elem * ns * p.nx;
    }
    case FDTD_READ_ETABLE: return (int64_t)sizeof(cd) * p.nt;
    case FDTD_READ_ROWS_DONE: return (int64_t)sizeof(int64_t);
  }
  return -1;
}

fdtd_status fdtd_readout(fdtd_plan_t P, int32_t kind, void* dst, int64_t dst_bytes) {
  if (!P) return FDTD_ERR_INVALID_ARG;
  if (P->state < 2) return fail(P, FDTD_ERR_STATE, "fdtd_readout before fdtd_set_boundary");
  if (P->batched) return batch_readout(P, 0, kind, dst, dst_bytes);
  int64_t need = fdtd_readout_bytes(P, kind);
  if (need < 0) return fail(P, FDTD_ERR_INVALID_ARG, "unknown readout kind");
  if (!dst || dst_bytes < need) return fail(P, FDTD_ERR_INVALID_ARG, "readout destination missing or too small");
  cudaError_t e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) return cuda_fail(P, e, "cudaStreamSynchronize");
  fdtd::SyncWords sw;
  e = cudaMemcpy(&sw, P->ws + P->off_sync, sizeof sw, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemcpy(status)");
  if (sw.status != 0) {
    char buf[128];
    snprintf(buf, sizeof buf, "device latched status %u (%s) at row %lld", sw.status,
             fdtd_status_string((fdtd_status)sw.status), (long long)sw.where);
    return fail(P, (fdtd_status)sw.status, buf);
  }
  const fdtd_params& p = P->p;
  const void* src = nullptr;
  switch (kind) {
    case FDTD_READ_ROW: src = P->ws + P->off_ring + P->elem * (size_t)((P->rows_done - 1) % P->R) * P->stride; break;
    case FDTD_READ_NORMS: src = P->ws + P->off_norms; break;
    case FDTD_READ_SNAPSHOTS: src = P->ws + P->off_snaps; break;
    case FDTD_READ_ETABLE: src = P->ws + P->off_etab; break;
    case FDTD_READ_ROWS_DONE: memcpy(dst, &P->rows_done, sizeof(int64_t)); return FDTD_OK;
  }
  if (need > 0) {
    e = cudaMemcpyAsync(dst, src, (size_t)need, cudaMemcpyDefault, P->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemcpyAsync(readout)");
  }
  (void)p;
  return FDTD_OK;
}

int64_t fdtd_readout_instance_bytes(fdtd_plan_t P, int32_t instance, int32_t kind) {
  if (!P) return -1;
  if (!P->batched) return instance == 0 ? fdtd_readout_bytes(P, kind) : -1;
  return batch_readout_bytes(P, instance, kind);
}

fdtd_status fdtd_readout_instance(fdtd_plan_t P, int32_t instance, int32_t kind, void* dst, int64_t dst_bytes) {
  if (!P) return FDTD_ERR_INVALID_ARG;
  if (P->state < 2) return fail(P, FDTD_ERR_STATE, "fdtd_readout_instance before fdtd_set_boundary");
  if (!P->batched) {
    if (instance != 0) return fail(P, FDTD_ERR_INVALID_ARG, "instance out of range");
    return fdtd_readout(P, kind, dst, dst_bytes);
  }
  return batch_readout(P, instance, kind, dst, dst_bytes);
}

void fdtd_destroy(fdtd_plan_t P) { delete P; }

fdtd_status fdtd_gamma_star(const int32_t* n, const double* z, double* out, int64_t count, void* cuda_stream) {
  if (count < 0 || (count > 0 && (!n || !z || !out))) return FDTD_ERR_INVALID_ARG;
  cudaError_t e = fdtd::launch_gamma_star(n, z, out, count, reinterpret_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? FDTD_OK : FDTD_ERR_CUDA;
}

}  // extern "C"
