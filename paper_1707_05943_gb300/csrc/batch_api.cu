// batch_api.cu -- host side of complex64 plans (FDTD_F32_COMP): one instance or
// a batch of independent instances marched by one persistent cluster launch.
// The boundary of every instance is built by the FP64 kernels of boundary.cu;
// the march reads FP32 copies of its tables.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "fdtd_internal.cuh"

using fdtd::cd;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

cd cdiv(cd a, cd b) {
  double d = b.re * b.re + b.im * b.im;
  return cd{(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

fdtd_status fail(fdtd_plan_s* p, fdtd_status s, const char* msg) {
  if (p && p->record_errors) p->last_error = msg;
  return s;
}
fdtd_status cuda_fail(fdtd_plan_s* p, cudaError_t e, const char* where) {
  if (p && p->record_errors) {
    p->last_error = where;
    p->last_error += ": ";
    p->last_error += cudaGetErrorString(e);
  }
  return FDTD_ERR_CUDA;
}

// gang share of complex64 plans (mid_weight): an instance is split into one band
// stream per total / (grid share / 8) updates of its own
constexpr int kGangShare = 16;
constexpr int kGangDefault = 32;  // band streams of the largest instance
constexpr int kTablePad = 64;     // zero entries beyond the sweep's reach (>= 32 + 8 + prefetch distance)
constexpr long long kSpinDefault = 4000000000LL;  // about 2 s at GB300 clocks

fdtd_status validate(const fdtd_params& p) {
  if (p.struct_size != sizeof(fdtd_params)) return FDTD_ERR_INVALID_ARG;
  if (p.D < 2 || (p.D & 1) || p.nx < p.D || p.nt < 1) return FDTD_ERR_INVALID_ARG;
  if (!(p.delta > 0) || !(p.gamma > 0) || !isfinite(p.omega0) || !isfinite(p.k)) return FDTD_ERR_INVALID_ARG;
  if (p.init_cond == FDTD_IC_TWO_PHOTON_PAIR) return FDTD_ERR_UNSUPPORTED;  // FP64-accurate plans only
  if (p.init_cond < FDTD_IC_PLANE_WAVE || p.init_cond > FDTD_IC_TWO_PHOTON_GAUSS) return FDTD_ERR_INVALID_ARG;
  if ((p.init_cond == FDTD_IC_STIM_EMISSION || p.init_cond == FDTD_IC_TWO_PHOTON_EXP) && !(p.alpha > 0))
    return FDTD_ERR_INVALID_ARG;
  if (p.init_cond == FDTD_IC_TWO_PHOTON_GAUSS && !(p.sigma > 0)) return FDTD_ERR_INVALID_ARG;
  if (p.tstep < -1 || p.rows_per_launch < 0 || p.spin_cycles < 0) return FDTD_ERR_INVALID_ARG;
  if (p.cluster_ctas < 0 || p.cluster_ctas > fdtd::kGangMax || p.mid_weight < 0 || p.mid_weight > 4096)
    return FDTD_ERR_INVALID_ARG;
  if (p.precision != FDTD_F32_COMP) return FDTD_ERR_INVALID_ARG;
  return FDTD_OK;
}

template <class T>
T* at(fdtd_plan_s* P, size_t off) {
  return reinterpret_cast<T*>(P->ws + off);
}

}  // namespace

fdtd::RowMap row_map(fdtd_plan_s* P, int i) {
  const fdtd_batch_inst& b = P->inst[i];
  fdtd::RowMap m;
  m.ring = at<float2>(P, b.off_ring);
  m.stride = b.stride;
  m.skew = at<float2>(P, b.off_skew);
  m.rd = b.p.nx - b.p.D;
  m.nx = b.p.nx;
  m.R = b.R;
  m.D = b.p.D;
  return m;
}

fdtd_status batch_plan_fill(fdtd_plan_s* P, const fdtd_params* pin, int32_t n, void* cuda_stream,
                            size_t* workspace_bytes) {
  if (n < 1) return FDTD_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    fdtd_status st = validate(pin[i]);
    if (st != FDTD_OK) return st;
  }
  P->batched = true;
  P->p = pin[0];
  P->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&P->device) != cudaSuccess) return FDTD_ERR_CUDA;
  cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
  P->record_errors = true;
  P->inst.assign(n, fdtd_batch_inst{});
  // the persistent launch: every CTA resident
  const int per_sm = fdtd::march_f32c_blocks_per_sm();
  if (per_sm <= 0) return FDTD_ERR_CUDA;
  P->grid = per_sm * P->num_sms;
  // gang (band streams in flight) of each instance: its share of the work in units
  // of total / (grid share/8), at most gang_max, at most its bands, and at most the
  // grid (no stream may wait on one that no CTA is free to take)
  P->gang_max = pin[0].cluster_ctas > 0 ? pin[0].cluster_ctas : kGangDefault;
  if (P->gang_max > P->grid) P->gang_max = P->grid;
  P->mid_weight = pin[0].mid_weight > 0 ? pin[0].mid_weight : kGangShare;
  double utot = 0.0;
  for (int i = 0; i < n; ++i) utot += (double)pin[i].nx * (double)pin[i].nt;
  const double unit = utot / ((double)P->grid * P->mid_weight / 8.0);

  size_t off = 0;
  P->off_sync = off;  off = align_up(off + sizeof(fdtd::SyncWords));
  P->off_desc = off;  off = align_up(off + sizeof(fdtd::InstDesc) * (size_t)n);
  P->off_order = off; off = align_up(off + sizeof(fdtd::WorkItem) * (size_t)n * fdtd::kGangMax);
  P->off_queue = off; off = align_up(off + sizeof(unsigned int) * 4);
  P->off_eargs = off; off = align_up(off + sizeof(fdtd::EtabArgs) * (size_t)n);
  for (int i = 0; i < n; ++i) {
    const fdtd_params& p = pin[i];
    fdtd_batch_inst& b = P->inst[i];
    b.p = p;
    const cd W = cd{0.5 * p.gamma, p.omega0};
    const cd A = cd{1.0 / p.delta + W.re / 4.0, W.im / 4.0};
    const cd B = cd{1.0 / p.delta - W.re / 4.0, -W.im / 4.0};
    b.cs = cdiv(cd{1.0, 0.0}, A);
    b.c1 = cdiv(B, A);
    b.c2 = cdiv(cd{-W.re / 4.0, -W.im / 4.0}, A);
    b.c3 = (p.gamma / 8.0) * b.cs;
    b.gs = (-p.gamma / 4.0) * b.cs;
    b.C = (p.init_cond == FDTD_IC_STIM_EMISSION) ? 1.0 : sqrt(2.0);
    // the row recurrence y_m = c2 y_{m-1} + r_m is stable only for |c2| < 1
    if (hypot(b.c2.re, b.c2.im) >= 1.0) return FDTD_ERR_UNSUPPORTED;
    const int64_t bands = (p.nt - 1 + fdtd::kF32Band - 1) / fdtd::kF32Band;
    int64_t g = (int64_t)ceil((double)p.nx * (double)p.nt / unit);
    g = std::min<int64_t>(std::min<int64_t>(g, P->gang_max), std::max<int64_t>(bands, 1));
    b.g = (int)std::max<int64_t>(g, 1);
    // rows an in-flight band reads: back to D + 1 below the oldest of g bands in flight
    b.R = p.D + 2 + fdtd::kF32Band * b.g + fdtd::kRowSlack;
    b.stride = (p.D + 31) / 32 * 32 + 32;  // inner ring row pitch (columns < D)
    b.nphi = p.nt + 3 * (int64_t)p.D + 8;
    b.nsnap = (p.tstep >= 0) ? (p.nt - 1) / (p.tstep + 1) + 1 : 0;
    b.dpad = (p.D + 7) / 8 * 8;
    b.nxpad = (p.nx + 7) / 8 * 8;
    b.lo_elems = 2 * b.dpad + b.nxpad + p.nt;
    b.off_etab = off;     off = align_up(off + sizeof(cd) * (size_t)p.nt);
    b.off_phi = off;      off = align_up(off + sizeof(cd) * (size_t)b.nphi);
    b.off_rowscal = off;  off = align_up(off + 2 * sizeof(cd) * (size_t)p.nt);
    b.off_detab = off;    off = align_up(off + sizeof(cd) * (size_t)(p.nt + p.D));
    b.off_norms = off;    off = align_up(off + sizeof(double) * (size_t)p.nt);
    b.off_hscr = off;     off = align_up(off + sizeof(cd) * (size_t)p.nt);
    b.off_etab32 = off;   off = align_up(off + sizeof(float2) * (size_t)p.nt);
    // FP32 source tables padded with zeros on both sides: the sweep walks them without
    // bounds tests (an index below 0, out of the light cone, gives 0)
    b.padl_e = (p.nx - p.D) + kTablePad;
    b.padl_f = (p.nx - p.D) + p.D + kTablePad;
    b.off_phi32 = off;    off = align_up(off + sizeof(float2) * (size_t)(b.padl_f + b.nphi + kTablePad));
    b.off_rowscal32 = off; off = align_up(off + 2 * sizeof(float2) * (size_t)p.nt);
    b.off_detab32 = off;  off = align_up(off + sizeof(float2) * (size_t)(b.padl_e + p.nt + p.D + kTablePad));
    b.off_lo = off;       off = align_up(off + sizeof(float2) * (size_t)b.lo_elems);
    b.off_bnd = off;      off = align_up(off + sizeof(float2) * 2 * (size_t)p.nt);
    b.off_bnorm = off;    off = align_up(off + sizeof(double) * (size_t)p.nt);
    b.off_bsync = off;    off = align_up(off + sizeof(unsigned long long) * (1 + fdtd::kGangMax));
    b.off_ring = off;     off = align_up(off + sizeof(float2) * (size_t)b.R * (size_t)b.stride);
    b.off_skew = off;     off = align_up(off + sizeof(float2) * (size_t)b.R * (size_t)(p.nx - p.D));
    b.off_snaps = off;    off = align_up(off + sizeof(float2) * (size_t)b.nsnap * (size_t)p.nx);
    b.rows_done = 0;
  }
  // one row of the widest instance: row readouts and checkpoints gather through it
  int64_t maxnx = 0;
  for (int i = 0; i < n; ++i) maxnx = std::max<int64_t>(maxnx, pin[i].nx);
  P->off_stage = off; off = align_up(off + sizeof(float2) * (size_t)maxnx);
  P->ws_need = off;
  P->state = 0;
  *workspace_bytes = off;
  return FDTD_OK;
}

fdtd_status batch_set_boundary(fdtd_plan_s* P, int32_t source, const void* table, int64_t ntab) {
  const int n = (int)P->inst.size();
  if (source != FDTD_BOUNDARY_ANALYTIC && source != FDTD_BOUNDARY_TABLE && source != FDTD_BOUNDARY_RESTORE)
    return fail(P, FDTD_ERR_INVALID_ARG, "unknown boundary source");
  if (source == FDTD_BOUNDARY_RESTORE && (!table || ntab <= 0))
    return fail(P, FDTD_ERR_INVALID_ARG, "checkpoint missing");
  int64_t total_nt = 0;
  for (auto& b : P->inst) total_nt += b.p.nt;
  if (source == FDTD_BOUNDARY_TABLE && (!table || ntab != total_nt))
    return fail(P, FDTD_ERR_INVALID_ARG, "boundary table must hold sum(nt) complex128 values");
  cudaStream_t s = P->stream;
  cudaError_t e = cudaMemsetAsync(P->ws + P->off_sync, 0, sizeof(fdtd::SyncWords), s);
  if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemsetAsync");
  std::vector<fdtd::InstDesc> desc(n);
  std::vector<fdtd::BoundaryArgs> bargs(n);
  std::vector<fdtd::EtabArgs> eargs(n);
  int64_t max_nt = 0;
  const char* tab = static_cast<const char*>(table);
  for (int i = 0; i < n; ++i) {
    fdtd_batch_inst& b = P->inst[i];
    const fdtd_params& p = b.p;
    // every ring row a march reads was written by it, except row 0 (zero at x > -a)
    e = fdtd::launch_row_move(row_map(P, i), 0, nullptr, 2, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->ws + b.off_norms, 0, sizeof(double) * (size_t)p.nt, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->ws + b.off_lo, 0, sizeof(float2) * (size_t)b.lo_elems, s);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(P->ws + b.off_bsync, 0, sizeof(unsigned long long) * (1 + fdtd::kGangMax), s);
    if (e == cudaSuccess && b.nsnap)
      e = cudaMemsetAsync(P->ws + b.off_snaps, 0, sizeof(float2) * (size_t)b.nsnap * (size_t)p.nx, s);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(P->ws + b.off_phi32, 0, sizeof(float2) * (size_t)(b.padl_f + b.nphi + kTablePad), s);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(P->ws + b.off_detab32, 0, sizeof(float2) * (size_t)(b.padl_e + p.nt + p.D + kTablePad), s);
    if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemsetAsync");
    if (source == FDTD_BOUNDARY_TABLE) {
      e = cudaMemcpyAsync(P->ws + b.off_etab, tab, sizeof(cd) * (size_t)p.nt, cudaMemcpyDeviceToDevice, s);
      tab += sizeof(cd) * (size_t)p.nt;
      if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemcpyAsync(table)");
    }
    fdtd::BoundaryArgs a;
    memset(&a, 0, sizeof a);  // no second photon: the pair fields stay null
    a.etab = at<cd>(P, b.off_etab);
    a.phitab = at<cd>(P, b.off_phi);
    a.rowscal = at<cd>(P, b.off_rowscal);
    a.detab = at<cd>(P, b.off_detab);
    a.norms = at<double>(P, b.off_norms);
    a.nt = p.nt;
    a.nphi = b.nphi;
    a.D = p.D;
    a.init_cond = p.init_cond;
    a.delta = p.delta;
    a.gamma = p.gamma;
    a.omega0 = p.omega0;
    a.k = p.k;
    a.alpha = p.alpha;
    a.sigma = p.sigma;
    a.center = p.center;
    a.C = b.C;
    a.cs = b.cs;
    a.status = &at<fdtd::SyncWords>(P, P->off_sync)->status;
    e = fdtd::launch_boundary_pre(a, s);
    if (e != cudaSuccess) return cuda_fail(P, e, "boundary kernels");
    bargs[i] = a;
    eargs[i] = fdtd::etable_args(a, at<cd>(P, b.off_hscr));
    max_nt = std::max<int64_t>(max_nt, p.nt);
  }
  // e(t) of every instance in one launch per pass (FP64)
  if (source != FDTD_BOUNDARY_TABLE) {
    e = cudaMemcpyAsync(P->ws + P->off_eargs, eargs.data(), sizeof(fdtd::EtabArgs) * (size_t)n,
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = fdtd::launch_etable_batch(at<fdtd::EtabArgs>(P, P->off_eargs), n, max_nt, s);
    if (e != cudaSuccess) return cuda_fail(P, e, "boundary e-tables");
  }
  for (int i = 0; i < n; ++i) {
    fdtd_batch_inst& b = P->inst[i];
    const fdtd_params& p = b.p;
    e = fdtd::launch_boundary_post(bargs[i], s);
    if (e != cudaSuccess) return cuda_fail(P, e, "boundary kernels");

    fdtd::InstDesc& d = desc[i];
    memset(&d, 0, sizeof d);
    d.nx = p.nx;
    d.nt = p.nt;
    d.stride = b.stride;
    d.nphi = b.nphi;
    d.range[0] = 1;
    d.range[1] = 1;
    d.D = p.D;
    d.R = b.R;
    d.tstep = p.tstep;
    auto f = [](cd v) { return make_float2((float)v.re, (float)v.im); };
    auto flo = [](cd v) {  // the part of v that its FP32 rounding drops
      return make_float2((float)(v.re - (double)(float)v.re), (float)(v.im - (double)(float)v.im));
    };
    const cd d1 = cd{b.c1.re - 1.0, b.c1.im};
    d.d1 = f(d1);
    d.c2 = f(b.c2);
    d.c3 = f(b.c3);
    d.d1lo = flo(d1);
    d.c2lo = flo(b.c2);
    d.c3lo = flo(b.c3);
    d.gs = f(b.gs);
    d.C = b.C;
    d.delta = p.delta;
    d.ring = at<float2>(P, b.off_ring);
    d.skew = at<float2>(P, b.off_skew);
    d.rd = p.nx - p.D;
    d.snaps = b.nsnap ? at<float2>(P, b.off_snaps) : nullptr;
    d.lo_in = at<float2>(P, b.off_lo);
    d.lo_row = d.lo_in + 2 * b.dpad;
    d.lo_edge = d.lo_row + b.nxpad;
    d.dpad = b.dpad;
    d.bsync = at<unsigned long long>(P, b.off_bsync);
    d.spin = p.spin_cycles > 0 ? (long long)p.spin_cycles : kSpinDefault;
    d.norms = at<double>(P, b.off_norms);
    d.etab = at<cd>(P, b.off_etab);
    d.phitab = at<cd>(P, b.off_phi);
    d.etab32 = at<float2>(P, b.off_etab32);
    d.phitab32 = at<float2>(P, b.off_phi32) + b.padl_f;
    d.detab32 = at<float2>(P, b.off_detab32) + b.padl_e;
    d.rowscal32 = at<float2>(P, b.off_rowscal32);
    d.bnd32 = at<float2>(P, b.off_bnd);
    d.bnorm = at<double>(P, b.off_bnorm);
    e = fdtd::launch_tables32(d, at<cd>(P, b.off_detab), at<cd>(P, b.off_rowscal), s);
    if (e != cudaSuccess) return cuda_fail(P, e, "tables32");
    b.rows_done = 1;
  }
  // the queue: largest instance first, each as its g band streams in order
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (double)P->inst[x].p.nx * (double)P->inst[x].p.nt > (double)P->inst[y].p.nx * (double)P->inst[y].p.nt;
  });
  std::vector<fdtd::WorkItem> items;
  for (int i : order)
    for (int r = 0; r < P->inst[i].g; ++r) items.push_back(fdtd::WorkItem{i, r, P->inst[i].g, 0});
  P->nitems = (int)items.size();
  if (source == FDTD_BOUNDARY_RESTORE) {
    // each instance resumes at its checkpoint's row (rings, remainders, norms loaded)
    std::vector<int64_t> done(n, 1);
    fdtd_status st = state_restore(P, table, ntab, s, done.data());
    if (st != FDTD_OK) {
      P->state = 1;
      return fail(P, st, "checkpoint does not match the plan's parameters, is cut short, or cannot be read");
    }
    for (int i = 0; i < n; ++i) desc[i].range[0] = desc[i].range[1] = done[i];
  }
  e = cudaMemcpyAsync(P->ws + P->off_desc, desc.data(), sizeof(fdtd::InstDesc) * (size_t)n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(P->ws + P->off_order, items.data(), sizeof(fdtd::WorkItem) * items.size(),
                        cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemcpyAsync(descriptors)");
  // the pageable copies above are staged before they return
  P->rows_done = P->inst[0].rows_done;
  P->state = 2;
  return FDTD_OK;
}

fdtd_status batch_march(fdtd_plan_s* P, int64_t rows) {
  const int n = (int)P->inst.size();
  int64_t maxleft = 0;
  for (auto& b : P->inst) maxleft = std::max<int64_t>(maxleft, b.p.nt - b.rows_done);
  if (rows > maxleft) rows = maxleft;
  if (rows <= 0) return FDTD_OK;
  const int64_t per = P->p.rows_per_launch > 0 ? P->p.rows_per_launch : 4096;
  cudaStream_t s = P->stream;
  for (int64_t done = 0; done < rows; done += per) {
    const int64_t step = std::min<int64_t>(per, rows - done);
    cudaError_t e = fdtd::launch_advance(at<fdtd::InstDesc>(P, P->off_desc), n, step, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->ws + P->off_queue, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess)
      e = fdtd::launch_march_f32c(at<fdtd::InstDesc>(P, P->off_desc), at<fdtd::WorkItem>(P, P->off_order), P->nitems,
                                  at<unsigned int>(P, P->off_queue), at<fdtd::SyncWords>(P, P->off_sync),
                                  P->grid, s);
    if (e != cudaSuccess) return cuda_fail(P, e, "march_f32c launch");
  }
  for (auto& b : P->inst) b.rows_done = std::min<int64_t>(b.p.nt, b.rows_done + rows);
  P->rows_done = P->inst[0].rows_done;
  return FDTD_OK;
}

// the same launches, recorded once per march length on an internal stream into a
// CUDA graph and replayed behind an event on the plan's stream
fdtd_status batch_march_graph(fdtd_plan_s* P, int64_t rows) {
  int64_t maxleft = 0;
  for (auto& b : P->inst) maxleft = std::max<int64_t>(maxleft, b.p.nt - b.rows_done);
  if (rows > maxleft) rows = maxleft;
  if (rows <= 0) return FDTD_OK;
  const int n = (int)P->inst.size();
  const int64_t per = P->p.rows_per_launch > 0 ? P->p.rows_per_launch : 4096;
  cudaError_t e = cudaSuccess;
  if (!P->cap_stream) {
    e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(P, e, "graph stream/events");
  }
  if (!P->graph_exec || P->graph_rows != rows) {
    if (P->graph_exec) {
      cudaGraphExecDestroy(P->graph_exec);
      P->graph_exec = nullptr;
    }
    cudaStream_t c = P->cap_stream;
    e = cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(P, e, "cudaStreamBeginCapture");
    for (int64_t done = 0; done < rows && e == cudaSuccess; done += per) {
      const int64_t step = std::min<int64_t>(per, rows - done);
      e = fdtd::launch_advance(at<fdtd::InstDesc>(P, P->off_desc), n, step, c);
      if (e == cudaSuccess) e = cudaMemsetAsync(P->ws + P->off_queue, 0, sizeof(unsigned int), c);
      if (e == cudaSuccess)
        e = fdtd::launch_march_f32c(at<fdtd::InstDesc>(P, P->off_desc), at<fdtd::WorkItem>(P, P->off_order),
                                    P->nitems, at<unsigned int>(P, P->off_queue), at<fdtd::SyncWords>(P, P->off_sync),
                                    P->grid, c);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&P->graph_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      P->graph_exec = nullptr;
      return cuda_fail(P, e, "graph capture");
    }
    P->graph_rows = rows;
  }
  e = cudaEventRecord(P->ev_in, P->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(P->cap_stream, P->ev_in, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(P->graph_exec, P->cap_stream);
  if (e == cudaSuccess) e = cudaEventRecord(P->ev_out, P->cap_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(P->stream, P->ev_out, 0);
  if (e != cudaSuccess) return cuda_fail(P, e, "graph launch");
  for (auto& b : P->inst) b.rows_done = std::min<int64_t>(b.p.nt, b.rows_done + rows);
  P->rows_done = P->inst[0].rows_done;
  return FDTD_OK;
}

int64_t batch_readout_bytes(fdtd_plan_s* P, int32_t i, int32_t kind) {
  if (i < 0 || i >= (int)P->inst.size()) return -1;
  const fdtd_batch_inst& b = P->inst[i];
  switch (kind) {
    case FDTD_READ_ROW: return (int64_t)sizeof(float2) * b.p.nx;
    case FDTD_READ_NORMS: return (int64_t)sizeof(double) * b.rows_done;
    case FDTD_READ_SNAPSHOTS: {
      if (!b.nsnap || b.rows_done == 0) return 0;
      int64_t ns = (b.rows_done - 1) / (b.p.tstep + 1) + 1;
      return (int64_t)sizeof(float2) * ns * b.p.nx;
    }
    case FDTD_READ_ETABLE: return (int64_t)sizeof(cd) * b.p.nt;
    case FDTD_READ_ROWS_DONE: return (int64_t)sizeof(int64_t);
    case FDTD_READ_STATE: return state_bytes(P, i);
  }
  return -1;
}

fdtd_status batch_readout(fdtd_plan_s* P, int32_t i, int32_t kind, void* dst, int64_t dst_bytes) {
  int64_t need = batch_readout_bytes(P, i, kind);
  if (need < 0) return fail(P, FDTD_ERR_INVALID_ARG, "unknown readout kind or instance");
  if (!dst || dst_bytes < need) return fail(P, FDTD_ERR_INVALID_ARG, "readout destination missing or too small");
  cudaError_t e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) return cuda_fail(P, e, "cudaStreamSynchronize");
  fdtd::SyncWords sw;
  e = cudaMemcpy(&sw, P->ws + P->off_sync, sizeof sw, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemcpy(status)");
  if (sw.status != 0) return fail(P, (fdtd_status)sw.status, "device latched an error");
  const fdtd_batch_inst& b = P->inst[i];
  const void* src = nullptr;
  switch (kind) {
    case FDTD_READ_ROW:
      e = fdtd::launch_row_move(row_map(P, i), b.rows_done - 1, at<float2>(P, P->off_stage), 0, P->stream);
      if (e != cudaSuccess) return cuda_fail(P, e, "row gather");
      src = P->ws + P->off_stage;
      break;
    case FDTD_READ_NORMS: src = P->ws + b.off_norms; break;
    case FDTD_READ_SNAPSHOTS: src = P->ws + b.off_snaps; break;
    case FDTD_READ_ETABLE: src = P->ws + b.off_etab; break;
    case FDTD_READ_ROWS_DONE: memcpy(dst, &b.rows_done, sizeof(int64_t)); return FDTD_OK;
    case FDTD_READ_STATE: {
      fdtd_status st = state_readout(P, i, dst, dst_bytes, P->stream);
      return st == FDTD_OK ? FDTD_OK : fail(P, st, "checkpoint copy");
    }
  }
  if (need > 0) {
    e = cudaMemcpyAsync(dst, src, (size_t)need, cudaMemcpyDefault, P->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemcpyAsync(readout)");
  }
  return FDTD_OK;
}
