// fdtd_api.cu -- host side of the C ABI declared in include/fdtd.h: parameter
// validation and derivation (Table 1, App. A/B), workspace layout, launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#include <new>
#include <vector>

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

// smallest k >= 1 with |x|^k < 2^-bits (x != 0), capped
int trunc_depth(double ax, int cap, int bits) {
  if (ax <= 0.0) return 1;
  if (ax >= 1.0) return cap + 1;
  double k = ceil(-(double)bits * log(2.0) / log(ax));
  if (k < 1) k = 1;
  return (k > cap) ? cap + 1 : (int)k;
}

template <class T>
T* at(fdtd_plan_t p, size_t off) {
  return reinterpret_cast<T*>(p->ws + off);
}

// Dependency lists of the row pipeline (RowDeps in fdtd_internal.cuh).  For each CTA b,
// every other CTA whose columns b reads, with the smallest lag at which it
// reads them (row n of b reads row n - lag of that CTA); and, transposed, the
// CTAs that read b.  The reads of a column j (buffer index) of row n:
//   j-1, j at lag 1 (stencil; the carry halo of khalo columns left of the
//   CTA's first column recomputes those columns too);
//   j-D-1, j-D at lag D (delay square, rows n-D and n-D-1);
//   for j < D: D-2-j, D-1-j at lag j+1 (mirror bar of line 2, row n-m-D/2);
//   for D <= j < 2D: 2D-2-j, 2D-1-j at lag j-D+1 (mirror bar of line 3,
//   row n-m+D/2).
// Columns outside [0, nx) are x <= -a (exact) and need nothing.
struct RowDepLists {
  std::vector<int> dep_off, rd_off, rd;
  std::vector<int2> dep;
};
RowDepLists build_row_deps(const int64_t* split, int G, int64_t nx, int D, int khalo) {
  auto owner = [&](int64_t col) {
    int lo = 0, hi = G;  // last b with split[b] <= col
    while (hi - lo > 1) {
      int mid = (lo + hi) / 2;
      if (split[mid] <= col) lo = mid; else hi = mid;
    }
    return lo;
  };
  RowDepLists d;
  d.dep_off.assign(G + 1, 0);
  std::vector<std::vector<int>> readers(G);
  for (int b = 0; b < G; ++b) {
    const int64_t jl = split[b], jh = split[b + 1];
    std::vector<int> best(G, INT32_MAX);
    if (jl < jh) {
      const int64_t h0 = jl - khalo > 0 ? jl - khalo : 0;
      auto mark_range = [&](int64_t c0, int64_t c1, int L) {  // columns [c0, c1)
        if (c0 < 0) c0 = 0;
        if (c1 > nx) c1 = nx;
        if (c0 >= c1) return;
        for (int o = owner(c0); o < G && split[o] < c1; ++o)
          if (split[o] < split[o + 1] && L < best[o]) best[o] = L;
      };
      mark_range(h0 - 1, jh, 1);
      mark_range(h0 - D - 1, jh - D, D);
      for (int64_t j = h0; j < jh && j < 2 * (int64_t)D; ++j) {
        if (j < D) mark_range(D - 2 - j, D - j, (int)(j + 1));
        else mark_range(2 * (int64_t)D - 2 - j, 2 * (int64_t)D - j, (int)(j - D + 1));
      }
    }
    for (int o = 0; o < G; ++o)
      if (o != b && best[o] != INT32_MAX) {
        d.dep.push_back(make_int2(o, best[o]));
        readers[o].push_back(b);
      }
    d.dep_off[b + 1] = (int)d.dep.size();
  }
  d.rd_off.assign(G + 1, 0);
  for (int b = 0; b < G; ++b) {
    for (int r : readers[b]) d.rd.push_back(r);
    d.rd_off[b + 1] = (int)d.rd.size();
  }
  return d;
}

// the second term's tables of a photon pair: e0, phi, R1'/R2', dE2, h scratch, and
// (double-float plans) the double-float copies of the first four
struct PairView {
  cd *etab2, *phitab2, *rowscal2, *detab2, *hscr2;
  float4* dw;  // C e0, phi, R1'/R2', dE2 (same layout as the first term's)
};
PairView pair_view(fdtd_plan_t P) {
  PairView v;
  memset(&v, 0, sizeof v);
  if (!P->off_pair) return v;
  const fdtd_params& p = P->p;
  cd* b = reinterpret_cast<cd*>(P->ws + P->off_pair);
  v.etab2 = b;
  v.phitab2 = v.etab2 + p.nt;
  v.rowscal2 = v.phitab2 + P->nphi;
  v.detab2 = v.rowscal2 + 2 * p.nt;
  v.hscr2 = v.detab2 + p.nt + p.D;
  if (P->dw)
    v.dw = reinterpret_cast<float4*>(
        P->ws + align_up(P->off_pair + sizeof(cd) * (size_t)(p.nt + P->nphi + 2 * p.nt + p.nt + p.D + p.nt) + 256));
  return v;
}

// the probe arrays in the workspace: row offsets, columns, output positions, values
struct ProbeView {
  int* off;
  int* col;
  int* idx;
  double2* val;
};
ProbeView probe_view(fdtd_plan_t P) {
  ProbeView v;
  v.off = reinterpret_cast<int*>(P->ws + P->off_probes);
  v.col = v.off + P->p.nt + 1;
  v.idx = v.col + P->p.max_probes;
  const size_t vb = align_up(sizeof(int) * (size_t)(P->p.nt + 1 + 2 * P->p.max_probes) + 16);
  v.val = reinterpret_cast<double2*>(P->ws + P->off_probes + vb);
  return v;
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
  if (p.init_cond < FDTD_IC_PLANE_WAVE || p.init_cond > FDTD_IC_TWO_PHOTON_PAIR) return FDTD_ERR_INVALID_ARG;
  if ((p.init_cond == FDTD_IC_STIM_EMISSION || p.init_cond == FDTD_IC_TWO_PHOTON_EXP ||
       p.init_cond == FDTD_IC_TWO_PHOTON_PAIR) && !(p.alpha > 0))
    return FDTD_ERR_INVALID_ARG;
  if (p.init_cond == FDTD_IC_TWO_PHOTON_PAIR && (!(p.alpha2 > 0) || !isfinite(p.k2))) return FDTD_ERR_INVALID_ARG;
  if (p.init_cond == FDTD_IC_TWO_PHOTON_GAUSS && !(p.sigma > 0)) return FDTD_ERR_INVALID_ARG;
  if (p.tstep < -1 || p.rows_per_launch < 0 || p.spin_cycles < 0) return FDTD_ERR_INVALID_ARG;
  if (p.cluster_ctas < 0 || p.cluster_ctas > 64 || p.mid_weight < 0 || p.mid_weight > 4096) return FDTD_ERR_INVALID_ARG;
  if (p.max_probes < 0 || p.max_probes > INT32_MAX || p.nt >= INT32_MAX) return FDTD_ERR_INVALID_ARG;
  if (p.precision != FDTD_F64 && p.precision != FDTD_F64_DW) return FDTD_ERR_UNSUPPORTED;

  P->p = p;
  P->dw = (p.precision == FDTD_F64_DW);
  P->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&P->device);
  if (e != cudaSuccess) return FDTD_ERR_CUDA;
  cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
  int maxg = P->dw ? fdtd::march_dw_max_grid(P->device) : fdtd::march_f64_max_grid(P->device);
  if (maxg <= 0) return FDTD_ERR_CUDA;
  // one CTA per SM (FDTD_F64_DW: every co-resident CTA), but at least 64 columns per CTA
  int grid = P->dw ? maxg : (P->num_sms < maxg ? P->num_sms : maxg);
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
  if (p.init_cond == FDTD_IC_TWO_PHOTON_PAIR) {
    // Sec. 2 (c): psi(x<=-a) = A [phi1 e0^(2) + phi2 e0^(1)] with the printed normalisation A
    const double dk = p.k - p.k2, sa = p.alpha + p.alpha2, G = p.gamma;
    const double num = 4.0 * dk * dk + sa * sa * G * G;
    P->C = sqrt(num / (num + 4.0 * p.alpha * p.alpha2 * G * G));
  }

  const double ac2 = cabsh(P->c2);
  // carries are exact while |c2|^k stays above the arithmetic's rounding:
  // 2^-60 in FP64, 2^-52 in double-float (48 significant bits)
  P->kfix = trunc_depth(ac2, fdtd::kMaxTrunc, P->dw ? 52 : 60);
  P->khalo = P->kfix;
  if (P->kfix > fdtd::kMaxTrunc)
    return FDTD_ERR_UNSUPPORTED;  // |c2| too close to 1 (delta far too coarse)

  // workspace layout
  P->R = p.D + 2 + fdtd::kRowSlack;
  P->rows_per_launch = p.rows_per_launch > 0 ? p.rows_per_launch : 4096;
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
  P->off_partials = off; off = align_up(off + sizeof(double) * (size_t)P->rows_per_launch * (size_t)grid);
  P->off_colsplit = off; off = align_up(off + sizeof(int64_t) * (size_t)(grid + 1));
  P->off_done = off;     off = align_up(off + sizeof(unsigned long long) * (size_t)grid);
  P->off_deps = off;     off = align_up(off + sizeof(int) * (size_t)(2 * (grid + 1) + 3 * fdtd::kMaxDeps));
  if (P->dw) {
    // double-float tables: C e (nt), phi (nphi), R1/R2 (2 nt), dE (nt + D)
    P->off_dwtab = off;  off = align_up(off + sizeof(float4) * (size_t)(4 * p.nt + P->nphi + p.D));
    P->off_rowout = off; off = align_up(off + sizeof(cd) * (size_t)p.nx);
  }
  if (p.init_cond == FDTD_IC_TWO_PHOTON_PAIR) {
    // second term: e0 (nt), phi (nphi), R1'/R2' (2 nt), dE2 (nt + D), h scratch (nt);
    // double-float copies of the first four
    P->off_pair = off;
    off = align_up(off + sizeof(cd) * (size_t)(p.nt + P->nphi + 2 * p.nt + p.nt + p.D + p.nt) + 256);
    if (P->dw) off = align_up(off + sizeof(float4) * (size_t)(4 * p.nt + P->nphi + p.D));
  }
  if (p.max_probes > 0) {  // row offsets (nt + 1), columns, output positions, values
    P->off_probes = off;
    off = align_up(off + sizeof(int) * (size_t)(p.nt + 1 + 2 * p.max_probes) + 16);
    off = align_up(off + sizeof(cd) * (size_t)p.max_probes);
    // chi points: up to max_probes / 4 records and their values
    P->off_chi = off;
    off = align_up(off + (sizeof(fdtd::ChiRec) + sizeof(cd)) * (size_t)(p.max_probes / 4 + 1));
  }
  if (p.init_cond == FDTD_IC_STIM_EMISSION) {
    P->off_e0tab = off;  off = align_up(off + sizeof(cd) * (size_t)p.nt);
    P->off_meas = off;   off = align_up(off + 4 * sizeof(double) * (size_t)P->nsnap);
  }
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
  if (source != FDTD_BOUNDARY_ANALYTIC && source != FDTD_BOUNDARY_TABLE && source != FDTD_BOUNDARY_RESTORE)
    return fail(P, FDTD_ERR_INVALID_ARG, "unknown boundary source");
  if (source == FDTD_BOUNDARY_TABLE && (!device_table || n != p.nt))
    return fail(P, FDTD_ERR_INVALID_ARG, "boundary table must hold nt complex128 values");
  if (source == FDTD_BOUNDARY_TABLE && p.init_cond == FDTD_IC_TWO_PHOTON_PAIR)
    return fail(P, FDTD_ERR_UNSUPPORTED, "a photon pair's boundary is computed, not given as a table");
  if (source == FDTD_BOUNDARY_RESTORE && (!device_table || n <= 0))
    return fail(P, FDTD_ERR_INVALID_ARG, "checkpoint missing");
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
  // (measured: a column of -a < x <= 3a costs ~16 bulk columns in FP64 and
  // ~20 in double-float, where the pipeline runs at the pace of its slowest CTA)
  const int kMidWeight = p.mid_weight > 0 ? p.mid_weight : (P->dw ? 20 : 16);
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
    // the double-float march runs every co-resident CTA: the pair sums must not
    // lower the CTAs that fit on an SM, else they are recomputed from the ring
    if (P->dw && P->march_smem &&
        (int64_t)fdtd::march_dw_blocks_per_sm(P->march_smem) * P->num_sms < P->grid)
      P->march_smem = 0;
  }
  e = cudaMemcpyAsync(P->ws + P->off_colsplit, split, sizeof(int64_t) * (size_t)(P->grid + 1), cudaMemcpyHostToDevice,
                      s);
  if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemcpyAsync(colsplit)");
  // a copy from pageable memory is staged before cudaMemcpyAsync returns
  fdtd::BoundaryArgs a;
  memset(&a, 0, sizeof a);
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
  const PairView pv = pair_view(P);
  a.etab2 = pv.etab2;
  a.phitab2 = pv.phitab2;
  a.rowscal2 = pv.rowscal2;
  a.detab2 = pv.detab2;
  a.k2 = p.k2;
  a.alpha2 = p.alpha2;
  if (p.init_cond == FDTD_IC_TWO_PHOTON_PAIR)
    e = fdtd::launch_boundary_pair(a, at<cd>(P, P->off_hscr), pv.hscr2, source != FDTD_BOUNDARY_TABLE, s);
  else
    e = fdtd::launch_boundary(a, at<cd>(P, P->off_hscr), source != FDTD_BOUNDARY_TABLE, s);
  if (e == cudaSuccess && p.init_cond == FDTD_IC_STIM_EMISSION)  // e0 of the measures (App. D)
    e = fdtd::launch_etable_e0(a, at<cd>(P, P->off_e0tab), at<cd>(P, P->off_hscr), s);
  if (e != cudaSuccess) return cuda_fail(P, e, "boundary kernels");
  if (P->dw) {
    float4* t = at<float4>(P, P->off_dwtab);
    e = fdtd::launch_tables_dw(a.etab, a.phitab, a.rowscal, a.detab, P->C, p.nt, P->nphi, p.D, t, t + p.nt,
                               t + p.nt + P->nphi, t + 3 * p.nt + P->nphi, s);
    if (e == cudaSuccess && pv.dw)
      e = fdtd::launch_tables_dw(pv.etab2, pv.phitab2, pv.rowscal2, pv.detab2, P->C, p.nt, P->nphi, p.D, pv.dw,
                                 pv.dw + p.nt, pv.dw + p.nt + P->nphi, pv.dw + 3 * p.nt + P->nphi, s);
    if (e != cudaSuccess) return cuda_fail(P, e, "double-float tables");
  }
  {
    // the row pipeline: row counters and the CTAs' dependency lists
    e = cudaMemsetAsync(P->ws + P->off_done, 0, sizeof(unsigned long long) * (size_t)P->grid, s);
    if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemsetAsync(row counters)");
    RowDepLists dd = build_row_deps(split, P->grid, p.nx, p.D, P->khalo);
    if ((int)dd.dep.size() > fdtd::kMaxDeps || (int)dd.rd.size() > fdtd::kMaxDeps)
      return fail(P, FDTD_ERR_UNSUPPORTED, "too many CTA dependencies for the row pipeline");
    // layout: dep_off[G+1] | rd_off[G+1] | dep (int2) | rd (int)
    std::vector<int> buf(2 * (P->grid + 1) + 3 * fdtd::kMaxDeps, 0);
    memcpy(buf.data(), dd.dep_off.data(), sizeof(int) * (P->grid + 1));
    memcpy(buf.data() + P->grid + 1, dd.rd_off.data(), sizeof(int) * (P->grid + 1));
    if (!dd.dep.empty()) memcpy(buf.data() + 2 * (P->grid + 1), dd.dep.data(), sizeof(int2) * dd.dep.size());
    if (!dd.rd.empty())
      memcpy(buf.data() + 2 * (P->grid + 1) + 2 * fdtd::kMaxDeps, dd.rd.data(), sizeof(int) * dd.rd.size());
    e = cudaMemcpyAsync(P->ws + P->off_deps, buf.data(), sizeof(int) * buf.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(P, e, "cudaMemcpyAsync(deps)");
  }
  P->rows_done = 1;
  P->n_probes = 0;
  P->n_chi = 0;
  if (source == FDTD_BOUNDARY_RESTORE) {
    int64_t done = 1;
    fdtd_status st = state_restore(P, device_table, n, s, &done);
    if (st != FDTD_OK) {
      P->state = 1;
      return fail(P, st, "checkpoint does not match the plan's parameters, is cut short, or cannot be read");
    }
    P->rows_done = done;
  }
  P->state = 2;
  return FDTD_OK;
}

static fdtd_status set_probes_impl(fdtd_plan_t P, const int64_t* points, int64_t count);

fdtd_status fdtd_set_probes(fdtd_plan_t P, const int64_t* points, int64_t count) {
  if (!P) return FDTD_ERR_INVALID_ARG;
  if (P->batched) return fail(P, FDTD_ERR_UNSUPPORTED, "probes need an FDTD_F64 or FDTD_F64_DW plan");
  if (P->state < 2) return fail(P, FDTD_ERR_STATE, "fdtd_set_probes before fdtd_set_boundary");
  P->n_chi = 0;
  return set_probes_impl(P, points, count);
}

// Eq. 2 at grid points (i1, i2, n): the four psi terms, each a probe of a
// marched point or the exact value of x <= -a, and the incident chi0.
fdtd_status fdtd_set_chi_points(fdtd_plan_t P, const int64_t* pts, int64_t count) {
  if (!P) return FDTD_ERR_INVALID_ARG;
  if (P->batched) return fail(P, FDTD_ERR_UNSUPPORTED, "chi needs an FDTD_F64 or FDTD_F64_DW plan");
  if (P->state < 2) return fail(P, FDTD_ERR_STATE, "fdtd_set_chi_points before fdtd_set_boundary");
  const fdtd_params& p = P->p;
  if (count < 0 || (count > 0 && !pts) || count > p.max_probes / 4)
    return fail(P, FDTD_ERR_INVALID_ARG, "chi point count negative or above max_probes / 4");
  const int64_t Dh = p.D / 2;
  auto theta = [](int64_t v) { return v > 0 ? 1.0 : (v == 0 ? 0.5 : 0.0); };
  std::vector<fdtd::ChiRec> recs((size_t)count);
  std::vector<int64_t> probes;
  probes.reserve((size_t)(4 * count));
  for (int64_t q = 0; q < count; ++q) {
    const int64_t i1 = pts[3 * q], i2 = pts[3 * q + 1], n = pts[3 * q + 2];
    if (n < 0 || n >= p.nt) return fail(P, FDTD_ERR_INVALID_ARG, "chi point row outside [0, nt)");
    fdtd::ChiRec& r = recs[q];
    memset(&r, 0, sizeof r);
    for (int sw = 0; sw < 2; ++sw) {
      const int64_t y1 = sw ? i2 : i1, y2 = sw ? i1 : i2;
      for (int side = 0; side < 2; ++side) {  // psi(y1-y2-+a, t-y2-+a) theta(y2+-a) theta(t-y2-+a)
        const int t = 2 * sw + side;
        const int64_t c = side ? y1 - y2 + Dh : y1 - y2 - Dh, row = side ? n - y2 + Dh : n - y2 - Dh;
        const double w = side ? -theta(y2 - Dh) * theta(row) : theta(y2 + Dh) * theta(row);
        r.w[t] = w;
        if (w == 0.0) continue;
        if (row >= p.nt) return fail(P, FDTD_ERR_INVALID_ARG, "chi point needs a row beyond nt");
        if (c <= -Dh) {  // x <= -a: C phi((c - row) delta) e(row delta)
          const int64_t ti = row - c - Dh;
          if (ti >= P->nphi) return fail(P, FDTD_ERR_INVALID_ARG, "chi point reaches past the wavepacket table");
          r.kind[t] = 2;
          r.idx[t] = (int32_t)ti;
          r.row[t] = (int32_t)row;
        } else {
          const int64_t j = c + Dh - 1;
          if (j >= p.nx) return fail(P, FDTD_ERR_INVALID_ARG, "chi point needs psi right of the marched box");
          if (row < P->rows_done && row > 0)
            return fail(P, FDTD_ERR_STATE, "chi point needs a row marched before the call");
          r.kind[t] = row == 0 ? 0 : 1;  // psi(x > -a, 0) = 0
          r.idx[t] = (int32_t)(probes.size() / 2);
          if (row > 0) {
            probes.push_back(row);
            probes.push_back(j);
          }
        }
      }
    }
    const int64_t f1 = n - i1 - Dh, f2 = n - i2 - Dh;  // phitab index of phi((i - n) delta) if x - t <= -a
    r.phi1 = (f1 >= 0 && f1 < P->nphi) ? (int32_t)f1 : -1;
    r.phi2 = (f2 >= 0 && f2 < P->nphi) ? (int32_t)f2 : -1;
    if ((f1 >= P->nphi) || (f2 >= P->nphi))
      return fail(P, FDTD_ERR_INVALID_ARG, "chi point reaches past the wavepacket table");
  }
  fdtd_status st = set_probes_impl(P, probes.data(), (int64_t)(probes.size() / 2));
  if (st != FDTD_OK) return st;
  if (count > 0) {
    cudaError_t e = cudaMemcpyAsync(P->ws + P->off_chi, recs.data(), sizeof(fdtd::ChiRec) * (size_t)count,
                                    cudaMemcpyHostToDevice, P->stream);
    if (e != cudaSuccess) return cuda_fail(P, e, "chi upload");
  }
  P->n_chi = count;
  return FDTD_OK;
}

static fdtd_status set_probes_impl(fdtd_plan_t P, const int64_t* points, int64_t count) {
  const fdtd_params& p = P->p;
  if (count < 0 || count > p.max_probes || (count > 0 && !points))
    return fail(P, FDTD_ERR_INVALID_ARG, "probe count negative or above max_probes");
  for (int64_t k = 0; k < count; ++k)
    if (points[2 * k] < 0 || points[2 * k] >= p.nt || points[2 * k + 1] < 0 || points[2 * k + 1] >= p.nx)
      return fail(P, FDTD_ERR_INVALID_ARG, "probe point outside the marched box");
  // by row: counting sort of the points, stable in the order given
  std::vector<int> off(p.nt + 1, 0), col(count > 0 ? count : 1), idx(count > 0 ? count : 1);
  for (int64_t k = 0; k < count; ++k) ++off[points[2 * k] + 1];
  for (int64_t n = 0; n < p.nt; ++n) off[n + 1] += off[n];
  std::vector<int> fill(off.begin(), off.end() - 1);
  for (int64_t k = 0; k < count; ++k) {
    const int q = fill[points[2 * k]]++;
    col[q] = (int)points[2 * k + 1];
    idx[q] = (int)k;
  }
  ProbeView v = probe_view(P);
  cudaStream_t s = P->stream;
  cudaError_t e = cudaMemcpyAsync(v.off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && count > 0)
    e = cudaMemcpyAsync(v.col, col.data(), sizeof(int) * (size_t)count, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && count > 0)
    e = cudaMemcpyAsync(v.idx, idx.data(), sizeof(int) * (size_t)count, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && count > 0) e = cudaMemsetAsync(v.val, 0, sizeof(double2) * (size_t)count, s);
  if (e != cudaSuccess) return cuda_fail(P, e, "probe upload");
  // the pageable copies are staged before cudaMemcpyAsync returns
  P->n_probes = count;
  return FDTD_OK;
}

fdtd_status fdtd_march_graph(fdtd_plan_t P, int64_t n_rows) {
  if (!P) return FDTD_ERR_INVALID_ARG;
  if (!P->batched) return fail(P, FDTD_ERR_UNSUPPORTED, "fdtd_march_graph needs an FDTD_F32_COMP plan");
  if (P->state < 2) return fail(P, FDTD_ERR_STATE, "fdtd_march_graph before fdtd_set_boundary");
  if (n_rows < 0) return fail(P, FDTD_ERR_INVALID_ARG, "n_rows < 0");
  return batch_march_graph(P, n_rows);
}

// the double-float march of rows [rows_done, end): one persistent launch per
// rows_per_launch rows, each followed by the FP64 norm reduction of its rows
static fdtd::RowDeps row_deps(fdtd_plan_t P) {
  int* deps = at<int>(P, P->off_deps);
  fdtd::RowDeps d;
  d.dep_off = deps;
  d.rd_off = deps + P->grid + 1;
  d.dep = reinterpret_cast<const int2*>(deps + 2 * (P->grid + 1));
  d.rd = deps + 2 * (P->grid + 1) + 2 * fdtd::kMaxDeps;
  d.done = at<unsigned long long>(P, P->off_done);
  return d;
}

static fdtd_status march_dw(fdtd_plan_t P, int64_t end) {
  const fdtd_params& p = P->p;
  fdtd::DwArgs a;
  memset(&a, 0, sizeof a);
  float4* t = at<float4>(P, P->off_dwtab);
  a.ring = at<float4>(P, P->off_ring);
  a.stride = P->stride;
  a.R = P->R;
  a.etabC = t;
  a.phitab = t + p.nt;
  a.rowscal = t + p.nt + P->nphi;
  a.detab = t + 3 * p.nt + P->nphi;
  const PairView pv = pair_view(P);
  if (pv.dw) {
    a.etabC2 = pv.dw;
    a.phitab2 = pv.dw + p.nt;
    a.rowscal2 = pv.dw + p.nt + P->nphi;
    a.detab2 = pv.dw + 3 * p.nt + P->nphi;
  }
  a.partials = at<double>(P, P->off_partials);
  a.snaps = P->nsnap ? at<double2>(P, P->off_snaps) : nullptr;
  a.colsplit = at<int64_t>(P, P->off_colsplit);
  a.deps = row_deps(P);
  a.sync = at<fdtd::SyncWords>(P, P->off_sync);
  a.nx = p.nx;
  a.nt = p.nt;
  a.nphi = P->nphi;
  a.D = p.D;
  a.tstep = p.tstep;
  a.kfix = P->kfix;
  a.khalo = P->khalo;
  a.hreuse = P->march_smem > 0 ? 1 : 0;
  a.mid_weight = P->mid_weight;
  auto split = [](cd v) {
    const float rh = (float)v.re, ih = (float)v.im;
    return make_float4(rh, ih, (float)(v.re - (double)rh), (float)(v.im - (double)ih));
  };
  a.d1 = split(cd{P->c1.re - 1.0, P->c1.im});
  a.c2 = split(P->c2);
  a.c3 = split(P->c3);
  a.gs = split(P->gs);
  cd pw = cd{1.0, 0.0};
  for (int k = 0; k <= fdtd::kMaxTrunc; ++k) {
    a.c2pow[k] = split(pw);
    pw = pw * P->c2;
  }
  a.spin_cycles = p.spin_cycles > 0 ? p.spin_cycles : 4000000000LL;  // default ~2 s at 2 GHz
  if (P->n_probes > 0) {
    ProbeView v = probe_view(P);
    a.probe_off = v.off;
    a.probe_col = v.col;
    a.probe_idx = v.idx;
    a.probe_val = v.val;
  }
  const int64_t per = P->rows_per_launch;
  for (int64_t n0 = P->rows_done; n0 < end; n0 += per) {
    a.n_begin = n0;
    a.n_end = (n0 + per < end) ? n0 + per : end;
    cudaError_t e = fdtd::launch_march_dw(a, P->grid, P->march_smem, P->stream);
    if (e == cudaSuccess)
      e = fdtd::launch_norms_rows(a.partials, P->grid, a.n_begin, a.n_end, at<cd>(P, P->off_etab),
                                  at<cd>(P, P->off_phi), pv.etab2, pv.phitab2, P->C, p.delta,
                                  at<double>(P, P->off_norms), P->stream);
    if (e != cudaSuccess) return cuda_fail(P, e, "double-float march launch");
  }
  P->rows_done = end;
  return FDTD_OK;
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
  if (P->dw) return march_dw(P, end);
  fdtd::MarchArgs a;
  memset(&a, 0, sizeof a);
  a.ring = at<cd>(P, P->off_ring);
  a.stride = P->stride;
  a.R = P->R;
  a.etab = at<cd>(P, P->off_etab);
  a.phitab = at<cd>(P, P->off_phi);
  a.rowscal = at<cd>(P, P->off_rowscal);
  a.detab = at<cd>(P, P->off_detab);
  {
    const PairView pv = pair_view(P);
    a.etab2 = pv.etab2;
    a.phitab2 = pv.phitab2;
    a.rowscal2 = pv.rowscal2;
    a.detab2 = pv.detab2;
  }
  a.norms = at<double>(P, P->off_norms);
  a.partials = at<double>(P, P->off_partials);
  a.snaps = P->nsnap ? at<cd>(P, P->off_snaps) : nullptr;
  a.colsplit = at<int64_t>(P, P->off_colsplit);
  a.deps = row_deps(P);
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
  a.spin_cycles = p.spin_cycles > 0 ? p.spin_cycles : 4000000000LL;  // default ~2 s at 2 GHz
  if (P->n_probes > 0) {
    ProbeView v = probe_view(P);
    a.probe_off = v.off;
    a.probe_col = v.col;
    a.probe_idx = v.idx;
    a.probe_val = v.val;
  }
  const int64_t per = P->rows_per_launch;
  for (int64_t n0 = P->rows_done; n0 < end; n0 += per) {
    a.n_begin = n0;
    a.n_end = (n0 + per < end) ? n0 + per : end;
    cudaError_t e = fdtd::launch_march_f64(a, P->grid, P->march_smem, P->stream);
    if (e == cudaSuccess)
      e = fdtd::launch_norms_rows(a.partials, P->grid, a.n_begin, a.n_end, a.etab, a.phitab, a.etab2, a.phitab2,
                                  P->C, p.delta, a.norms, P->stream);
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
    case FDTD_READ_STATE: return state_bytes(P, 0);
    case FDTD_READ_PROBES: return (int64_t)sizeof(cd) * P->n_probes;
    case FDTD_READ_CHI: return (int64_t)sizeof(cd) * P->n_chi;
    case FDTD_READ_MEASURES: {
      if (p.init_cond != FDTD_IC_STIM_EMISSION || !P->nsnap) return -1;
      if (P->rows_done == 0) return 0;
      int64_t ns = (P->rows_done - 1) / (p.tstep + 1) + 1;
      return (int64_t)(4 * sizeof(double)) * ns;
    }
  }
  return -1;
}

fdtd_status fdtd_readout(fdtd_plan_t P, int32_t kind, void* dst, int64_t dst_bytes) {
  if (!P) return FDTD_ERR_INVALID_ARG;
  if (P->state < 2) return fail(P, FDTD_ERR_STATE, "fdtd_readout before fdtd_set_boundary");
  if (P->batched) return batch_readout(P, 0, kind, dst, dst_bytes);
  int64_t need = fdtd_readout_bytes(P, kind);
  if (need < 0 && kind == FDTD_READ_MEASURES)
    return fail(P, FDTD_ERR_INVALID_ARG, "measures need a stimulated-emission plan with snapshots (tstep >= 0)");
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
    case FDTD_READ_ROW:
      src = P->ws + P->off_ring + P->elem * (size_t)((P->rows_done - 1) % P->R) * P->stride;
      if (P->dw) {  // double-float pairs -> complex128
        e = fdtd::launch_row_dw(static_cast<const float4*>(src), p.nx, at<double2>(P, P->off_rowout), P->stream);
        if (e != cudaSuccess) return cuda_fail(P, e, "row conversion");
        src = P->ws + P->off_rowout;
      }
      break;
    case FDTD_READ_NORMS: src = P->ws + P->off_norms; break;
    case FDTD_READ_SNAPSHOTS: src = P->ws + P->off_snaps; break;
    case FDTD_READ_ETABLE: src = P->ws + P->off_etab; break;
    case FDTD_READ_ROWS_DONE: memcpy(dst, &P->rows_done, sizeof(int64_t)); return FDTD_OK;
    case FDTD_READ_STATE: {
      fdtd_status st = state_readout(P, 0, dst, dst_bytes, P->stream);
      return st == FDTD_OK ? FDTD_OK : fail(P, st, "checkpoint copy");
    }
    case FDTD_READ_PROBES: src = probe_view(P).val; break;
    case FDTD_READ_CHI: {
      const fdtd::ChiRec* recs = at<fdtd::ChiRec>(P, P->off_chi);
      double2* vals = reinterpret_cast<double2*>(P->ws + P->off_chi + sizeof(fdtd::ChiRec) * (size_t)(p.max_probes / 4 + 1));
      const PairView pv = pair_view(P);
      e = fdtd::launch_chi(recs, P->n_chi, probe_view(P).val, at<cd>(P, P->off_phi), at<cd>(P, P->off_etab),
                           pv.phitab2, pv.etab2, P->C, p.gamma, p.init_cond != FDTD_IC_STIM_EMISSION, vals,
                           P->stream);
      if (e != cudaSuccess) return cuda_fail(P, e, "chi kernel");
      src = vals;
      break;
    }
    case FDTD_READ_MEASURES:
      e = fdtd::launch_measures(at<cd>(P, P->off_snaps), p.nx, p.tstep, need / (int64_t)(4 * sizeof(double)),
                                at<cd>(P, P->off_etab), at<cd>(P, P->off_e0tab), at<cd>(P, P->off_phi),
                                at<double>(P, P->off_norms), p.D, p.delta, p.gamma, p.alpha,
                                at<double>(P, P->off_meas), P->stream);
      if (e != cudaSuccess) return cuda_fail(P, e, "measures kernel");
      src = P->ws + P->off_meas;
      break;
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
