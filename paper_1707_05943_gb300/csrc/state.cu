// state.cu -- checkpoint and resume of a march (FDTD_READ_STATE and
// FDTD_BOUNDARY_RESTORE).  The paper's program keeps the whole grid; a march
// here keeps only the rows the update still reads (the delay term reaches row
// n-D-1), so a checkpoint is those rows plus what the readout has accumulated:
//
//   header (kStateHeaderBytes)                 parameters and counts, below
//   rows   rows_kept x nx x elem_bytes          rows rows_done-rows_kept .. rows_done-1,
//                                               row-major in the plan's own element
//                                               format (complex128, double-float pairs
//                                               or complex64), so that a resumed march
//                                               is bitwise the uninterrupted one (a
//                                               complex64 row is gathered from its two
//                                               rings through the plan's staging row)
//   lo     lo_elems x 8 B (complex64 only)      the TwoSum remainders the next row adds
//                                               along its characteristics: inner columns
//                                               (two row slots), the other columns of the
//                                               last row, column D-1 of every row
//   norms  rows_done x 8 B                      N(n) of every row so far
//
// A batched plan's checkpoint is one such record per instance, back to back.
// The boundary tables are not stored: RESTORE rebuilds them from the
// parameters.  Snapshots are not part of the state.
#include <cuda_runtime.h>
#include <string.h>

#include <vector>

#include "fdtd_internal.cuh"

using fdtd::cd;

namespace {

constexpr uint32_t kStateMagic = 0x53544446u;  // "FDTS"
constexpr uint32_t kStateVersion = 2;
constexpr size_t kStateHeaderBytes = 256;

struct StateHeader {
  uint32_t magic, version;
  int32_t precision, D;
  int64_t nx, nt, rows_done, rows_kept, lo_elems;
  int32_t elem_bytes, init_cond;
  double delta, gamma, omega0, k, alpha, sigma, center, k2, alpha2;
};
static_assert(sizeof(StateHeader) <= kStateHeaderBytes, "state header");

// the storage of one instance, whichever kind of plan holds it
struct InstView {
  const fdtd_params* p;
  char* ring;
  int64_t stride, R;
  size_t elem;
  char* lo;  // complex64 only
  int64_t lo_elems;
  double* norms;
  int64_t* rows_done;
  bool gathered;  // complex64: rows are spread over two rings; copied through P's staging row
};

InstView view(fdtd_plan_s* P, int i) {
  InstView v;
  if (P->batched) {
    fdtd_batch_inst& b = P->inst[i];
    v.p = &b.p;
    v.ring = P->ws + b.off_ring;
    v.stride = b.stride;
    v.R = b.R;
    v.elem = sizeof(float2);
    v.lo = P->ws + b.off_lo;
    v.lo_elems = b.lo_elems;
    v.norms = reinterpret_cast<double*>(P->ws + b.off_norms);
    v.rows_done = &b.rows_done;
    v.gathered = true;
  } else {
    v.p = &P->p;
    v.ring = P->ws + P->off_ring;
    v.stride = P->stride;
    v.R = P->R;
    v.elem = P->elem;
    v.lo = nullptr;
    v.lo_elems = 0;
    v.norms = reinterpret_cast<double*>(P->ws + P->off_norms);
    v.rows_done = &P->rows_done;
    v.gathered = false;
  }
  return v;
}

int64_t rows_kept(const InstView& v, int64_t rows_done) {
  const int64_t keep = (int64_t)v.p->D + 2;
  return rows_done < keep ? rows_done : keep;
}

int64_t record_bytes(const InstView& v, int64_t rows_done) {
  return (int64_t)kStateHeaderBytes + rows_kept(v, rows_done) * v.p->nx * (int64_t)v.elem +
         v.lo_elems * (int64_t)sizeof(float2) + rows_done * (int64_t)sizeof(double);
}

}  // namespace

int64_t state_bytes(fdtd_plan_s* P, int inst) {
  if (P->batched && (inst < 0 || inst >= (int)P->inst.size())) return -1;
  InstView v = view(P, P->batched ? inst : 0);
  return record_bytes(v, *v.rows_done);
}

// copy instance `inst`'s record into dst (any memory); the stream is synchronised
fdtd_status state_readout(fdtd_plan_s* P, int inst, void* dst, int64_t dst_bytes, cudaStream_t s) {
  if (!P->batched) inst = 0;
  InstView v = view(P, inst);
  const int64_t done = *v.rows_done;
  const int64_t need = record_bytes(v, done);
  if (!dst || dst_bytes < need) return FDTD_ERR_INVALID_ARG;
  unsigned char hb[kStateHeaderBytes];
  memset(hb, 0, sizeof hb);
  StateHeader h;
  memset(&h, 0, sizeof h);
  h.magic = kStateMagic;
  h.version = kStateVersion;
  h.precision = v.p->precision;
  h.D = v.p->D;
  h.nx = v.p->nx;
  h.nt = v.p->nt;
  h.rows_done = done;
  h.rows_kept = rows_kept(v, done);
  h.lo_elems = v.lo_elems;
  h.elem_bytes = (int32_t)v.elem;
  h.init_cond = v.p->init_cond;
  h.delta = v.p->delta;
  h.gamma = v.p->gamma;
  h.omega0 = v.p->omega0;
  h.k = v.p->k;
  h.alpha = v.p->alpha;
  h.sigma = v.p->sigma;
  h.center = v.p->center;
  h.k2 = v.p->k2;
  h.alpha2 = v.p->alpha2;
  memcpy(hb, &h, sizeof h);
  char* d = static_cast<char*>(dst);
  cudaError_t e = cudaMemcpyAsync(d, hb, kStateHeaderBytes, cudaMemcpyDefault, s);
  d += kStateHeaderBytes;
  const size_t row_bytes = v.elem * (size_t)v.p->nx;
  for (int64_t r = done - h.rows_kept; r < done && e == cudaSuccess; ++r) {
    if (v.gathered) {
      float2* stage = reinterpret_cast<float2*>(P->ws + P->off_stage);
      e = fdtd::launch_row_move(row_map(P, inst), r, stage, 0, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d, stage, row_bytes, cudaMemcpyDefault, s);
    } else {
      e = cudaMemcpyAsync(d, v.ring + v.elem * (size_t)((r % v.R) * v.stride), row_bytes, cudaMemcpyDefault, s);
    }
    d += row_bytes;
  }
  if (v.lo_elems && e == cudaSuccess) {
    e = cudaMemcpyAsync(d, v.lo, sizeof(float2) * (size_t)v.lo_elems, cudaMemcpyDefault, s);
    d += sizeof(float2) * (size_t)v.lo_elems;
  }
  if (e == cudaSuccess && done > 0) e = cudaMemcpyAsync(d, v.norms, sizeof(double) * (size_t)done, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // hb is on this stack frame
  return e == cudaSuccess ? FDTD_OK : FDTD_ERR_CUDA;
}

// Load the records at blob (any memory, nbytes) into the plan's instances, after
// the boundary tables have been rebuilt; sets each instance's rows_done.
// Errors: FDTD_ERR_INVALID_ARG (a record that does not match the plan or is
// cut short), FDTD_ERR_CUDA.
fdtd_status state_restore(fdtd_plan_s* P, const void* blob, int64_t nbytes, cudaStream_t s, int64_t* rows_restored) {
  const int n = P->batched ? (int)P->inst.size() : 1;
  const char* src = static_cast<const char*>(blob);
  int64_t left = nbytes;
  for (int i = 0; i < n; ++i) {
    InstView v = view(P, i);
    if (left < (int64_t)kStateHeaderBytes) return FDTD_ERR_INVALID_ARG;
    StateHeader h;
    if (cudaMemcpy(&h, src, sizeof h, cudaMemcpyDefault) != cudaSuccess) return FDTD_ERR_CUDA;
    const fdtd_params& p = *v.p;
    if (h.magic != kStateMagic || h.version != kStateVersion || h.precision != p.precision || h.D != p.D ||
        h.nx != p.nx || h.nt != p.nt || h.init_cond != p.init_cond || h.elem_bytes != (int32_t)v.elem ||
        h.lo_elems != v.lo_elems || h.delta != p.delta || h.gamma != p.gamma || h.omega0 != p.omega0 ||
        h.k != p.k || h.alpha != p.alpha || h.sigma != p.sigma || h.center != p.center || h.k2 != p.k2 ||
        h.alpha2 != p.alpha2)
      return FDTD_ERR_INVALID_ARG;
    if (h.rows_done < 1 || h.rows_done > p.nt || h.rows_kept != rows_kept(v, h.rows_done))
      return FDTD_ERR_INVALID_ARG;
    const int64_t rec = record_bytes(v, h.rows_done);
    if (left < rec) return FDTD_ERR_INVALID_ARG;
    const char* d = src + kStateHeaderBytes;
    const size_t row_bytes = v.elem * (size_t)p.nx;
    cudaError_t e = cudaSuccess;
    for (int64_t r = h.rows_done - h.rows_kept; r < h.rows_done && e == cudaSuccess; ++r) {
      if (v.gathered) {
        float2* stage = reinterpret_cast<float2*>(P->ws + P->off_stage);
        e = cudaMemcpyAsync(stage, d, row_bytes, cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = fdtd::launch_row_move(row_map(P, i), r, stage, 1, s);
      } else {
        e = cudaMemcpyAsync(v.ring + v.elem * (size_t)((r % v.R) * v.stride), d, row_bytes, cudaMemcpyDefault, s);
      }
      d += row_bytes;
    }
    if (v.lo_elems && e == cudaSuccess) {
      e = cudaMemcpyAsync(v.lo, d, sizeof(float2) * (size_t)v.lo_elems, cudaMemcpyDefault, s);
      d += sizeof(float2) * (size_t)v.lo_elems;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(v.norms, d, sizeof(double) * (size_t)h.rows_done, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return FDTD_ERR_CUDA;
    *v.rows_done = h.rows_done;
    rows_restored[i] = h.rows_done;
    src += rec;
    left -= rec;
  }
  // the copies read the caller's blob: finish them before returning
  return cudaStreamSynchronize(s) == cudaSuccess ? FDTD_OK : FDTD_ERR_CUDA;
}
