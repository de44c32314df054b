// march_f32c.cu -- complex64 march of Eq. 1 with a compensated increment, for
// one instance or a batch of independent instances in one persistent launch.
//
// The update is the FP64 one (march_f64.cu), split as
//   psi[n][m] = a + S,   a = psi[n-1][m-1],
//   S = d1 a + c2 (psi[n-1][m] + psi[n][m-1]) + c3 (delay square) + sources,
// with c1 = 1 + d1 (d1 = -(W/2)/A, |d1| ~ |W delta|/2).  S is O(|W delta|) |psi|
// and is formed in FP32.  The only term with weight ~1 is a, which is carried
// along its characteristic as an unevaluated pair a_hi + a_lo: a_hi is the
// complex64 value in the ring, a_lo the rounding error of the sum that
// produced it, recovered exactly by TwoSum(a_hi, S) (Knuth) and handed to the
// update of column m+1 of the next row.  The coefficients carry FP32 low parts
// (a coefficient error is the same at every step, so it would grow linearly
// along a characteristic).  The boundary tables, the exact boundary value
// psi(-a, t) at the first column and the norm reduction stay FP64.
//
// Work layout: bands of 256 consecutive rows, one row per thread.
//  * Inner columns -a < x <= a (storage columns j < D): the mirror term of
//    Eq. 1 reads row n-j-1 at column D-j-1, to the RIGHT of j, so these columns
//    go row by row: each thread takes a few columns, forms their sources, and
//    an exact affine scan over the threads (y -> c2^L y + Y per segment) gives
//    every segment its carry of the row recurrence y_m = c2 y_{m-1} + r_m.
//  * Columns x > a (j >= D): every read lies to the left or D rows back, so the
//    band sweeps them left to right as a systolic array: lane l of warp w marches
//    row n0 + 32w + l one column per step, one column behind the lane above.
//    Row n-1's value, its TwoSum remainder and its delay pair sum reach the lane
//    from the lane above by warp shuffles; lane 0 takes them from the warp above
//    through a shared-memory queue, warp 0 from the previous band's last row in
//    global memory.  The recurrence along the row is the lane's own running
//    value: exact, with no carries and no barriers.  Each lane streams one new
//    delay value (row n-D) per step, prefetched two steps ahead.
// A band is one CTA.  Every CTA of the persistent (cooperative) launch takes band
// streams from a queue, largest instance first: an instance with gang size g
// (set on the host from its share of the work) is split into g streams, stream r
// marching bands r, r + g, r + 2g, ...; so up to g bands (256 g rows) of one
// instance are in flight.  Band c waits (bounded) for band c-1's inner columns
// before its own, and its warp 0 for band c-1's last row before each chunk of 32
// columns; a ring of D + 2 + 256 g + 32 rows keeps every row an in-flight band
// reads.  The results do not depend on how rows fall into bands: every value is
// formed by the same operations in the same order whichever band, warp or lane
// computes it.
#include <cuda_runtime.h>

#include "fdtd_internal.cuh"

namespace fdtd {

namespace {

constexpr int kBand = kF32Band;           // rows per band: one per thread
constexpr int kWarps = kF32Threads / 32;  // warps per band
constexpr int kHandQ = 64;                // queue entries between consecutive warps (power of two)
constexpr int kGrp = 8;                   // sweep steps between queue bookkeeping
constexpr int kChunk = 32;                // columns of the previous band's last row staged at a time
constexpr int kPre = 2;                   // prefetch distance (sweep steps) of a lane's streams
constexpr int kInnerPer = 8;              // inner columns per thread and pass (2048 per pass)
static_assert(kBand == kF32Threads, "one row per thread");
static_assert(kPre == 2 && kGrp % kPre == 0 && kChunk % kGrp == 0, "sweep step grouping");
static_assert(kHandQ >= 31 + 2 * kGrp + 16, "queue too short for the sweep's lag");

struct Hand {
  float2 hi, lo, hn;  // psi[n][j] (hi, TwoSum remainder) and the delay pair sum of row n-D
};

}  // namespace

// the march kernel's shared memory, at namespace scope so that every helper addresses
// it as shared memory (a pointer parameter would make each access a generic one)
__shared__ Hand s_queue[kWarps][kHandQ];  // lane 0's input of warp w: warp w-1's last row (w > 0)
                                          // or the previous band's last row (w = 0)
__shared__ int s_prod[kWarps], s_cons[kWarps];
__shared__ float2 s_pv_hi[2][kChunk], s_pv_lo[2][kChunk], s_pv_d[2][kChunk + 1];
__shared__ float s_wn[kWarps][kBand];
__shared__ float2 s_scP[kWarps], s_scY[kWarps];
__shared__ float2 s_ylast;
__shared__ int s_item;
__shared__ __align__(16) InstDesc s_I;  // the instance's descriptor: no global store can alias it

__device__ __forceinline__ float2 f2(float r, float i) { return make_float2(r, i); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return f2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return f2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mulc(float2 a, float2 b) { return f2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 fmac(float2 a, float2 b, float2 acc) {  // acc + a*b
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float2 scal(float s, float2 a) { return f2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 shfl_up2(float2 v, int d) {
  return f2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}

// 8-byte asynchronous copies global -> shared (completion by commit groups)
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// TwoSum: s = fl(a+b), e = (a+b) - s exactly (round to nearest, no FMA involved)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// psi at x <= -a (c <= -D/2): C phi(-a - (r - c - D/2) delta) e(r delta) from the FP32 tables
__device__ __forceinline__ float2 psi_left32(const InstDesc& I, int64_t r, int64_t c) {
  const int Dh = I.D >> 1;
  return scal((float)I.C, mulc(I.phitab32[r - c - Dh], I.etab32[r]));
}

// S without a_lo and the c2 y term, and a_hi, for an inner column 0 <= j < D of row n
// (m = j - D/2 + 1 <= D/2).  The delay square lies at x <= -a; the mirror bar of row
// r2 = n - j - 1 reads columns D-j-2, D-j-1 of the ring.
__device__ __forceinline__ float2 rhs_inner32(const InstDesc& I, int64_t n, int nslot, int64_t j, float2 R2,
                                              float2* a_hi) {
  const int D = I.D, Dh = D >> 1, R = I.R;
  const int64_t m = j - Dh + 1;
  int s1 = nslot - 1;
  if (s1 < 0) s1 += R;
  const float2* row1 = I.ring + (int64_t)s1 * I.stride;
  const float2 v0 = (j >= 1) ? row1[j - 1] : psi_left32(I, n - 1, m - 1);
  const float2 v1 = row1[j];
  const bool dl = (n >= D + 1);
  const int64_t r2 = n - j - 1;
  const bool s2 = (r2 >= 0);
  float2 v2 = f2(0.f, 0.f), v3 = v2, v4 = v2, v5 = v2, v6 = v2, v7 = v2, v8 = v2, v9 = v2, chi = v2;
  if (dl) {
    v2 = psi_left32(I, n - D, m - D);
    v3 = psi_left32(I, n - D, m - D - 1);
    v4 = psi_left32(I, n - D - 1, m - D);
    v5 = psi_left32(I, n - D - 1, m - D - 1);
  }
  if (s2) {
    int s = nslot - (int)(j + 1);
    if (s < 0) s += R;
    const float2* rowr = I.ring + (int64_t)s * I.stride;
    v6 = psi_left32(I, r2, -m - D);
    v7 = psi_left32(I, r2, -m - D + 1);
    v8 = (j < D - 1) ? rowr[D - 2 - j] : psi_left32(I, r2, -m);
    v9 = rowr[D - 1 - j];
    chi = I.phitab32[r2];
  }
  *a_hi = v0;
  float2 S = mulc(I.d1, v0);
  S = fmac(I.c2, v1, S);
  float2 L = mulc(I.d1lo, v0);
  L = fmac(I.c2lo, v1, L);
  if (dl) {
    const float2 sq = add(add(v2, v3), add(v4, v5));
    S = fmac(I.c3, sq, S);
    L = fmac(I.c3lo, sq, L);
  }
  S = add(S, L);
  if (s2) {
    const float w = (r2 == 0) ? 0.5f : 1.0f;
    S = fmac(I.gs, scal(w, sub(add(v6, v7), add(v8, v9))), S);
    S = fmac(R2, chi, S);
  }
  return S;
}

// the mirror terms of a column D <= j < 2D (a < x <= 3a) of row n, added to S: the
// bar of row r2 = n-j-1 lies at x <= -a; the bar of row r3 = r2 + D reads ring
// columns 2D-j-2, 2D-j-1 (inner columns) and the boundary tables
__device__ __noinline__ float2 general_extra32(int n, int nslot, int j, float2 R2, float2 S) {
  const InstDesc& I = s_I;
  const int D = I.D, Dh = D >> 1;
  const int m = j - Dh + 1;
  const int r2 = n - j - 1, r3 = r2 + D;
  if (r2 >= 0) {
    const float2 v6 = psi_left32(I, r2, -m - D), v7 = psi_left32(I, r2, -m - D + 1);
    const float2 v8 = psi_left32(I, r2, -m), v9 = psi_left32(I, r2, -m + 1);
    const float w = (r2 == 0) ? 0.5f : 1.0f;
    S = fmac(I.gs, scal(w, sub(add(v6, v7), add(v8, v9))), S);
    S = fmac(R2, I.phitab32[r2], S);
  }
  if (r3 >= 0) {
    int s = nslot - (j + 1 - D);
    if (s < 0) s += I.R;
    const float2* rowr = I.ring + (int64_t)s * I.stride;
    const float2 v10 = (j <= 2 * D - 2) ? rowr[2 * D - 2 - j] : psi_left32(I, r3, D - m);
    const float2 v11 = rowr[2 * D - 1 - j];
    const float2 v12 = psi_left32(I, r3, -m), v13 = psi_left32(I, r3, -m + 1);
    const float w = (r3 == 0) ? 0.5f : 1.0f;
    S = fmac(I.gs, scal(w, sub(add(v10, v11), add(v12, v13))), S);
  }
  return S;
}

__device__ __forceinline__ void latch_timeout(SyncWords* sync, int64_t n) {
  if (atomicCAS(&sync->status, 0u, (unsigned)FDTD_ERR_TIMEOUT) == 0u) sync->where = n;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(p) : "memory");
  return v;
}
// bounded waits: poll until *p >= target, giving up after `spin` cycles (latching
// FDTD_ERR_TIMEOUT) or as soon as an error is latched; the polls are relaxed, the
// final read an acquire (GPU scope) or a CTA fence (shared memory)
__device__ __noinline__ void wait_ge_global_slow(const unsigned long long* p, unsigned long long target,
                                                 long long spin, SyncWords* sync, int64_t n) {
  const long long t0 = clock64();
  for (int k = 1;; ++k) {
    __nanosleep(64);
    if (ld_relaxed_u64(p) >= target) return;
    if ((k & 15) == 0 && *(volatile unsigned int*)&sync->status != 0u) return;
    if (clock64() - t0 > spin) {
      latch_timeout(sync, n);
      return;
    }
  }
}
__device__ __forceinline__ void wait_ge_global(const unsigned long long* p, unsigned long long target, long long spin,
                                               SyncWords* sync, int64_t n) {
  if (ld_relaxed_u64(p) < target) wait_ge_global_slow(p, target, spin, sync, n);
  (void)ld_acquire_u64(p);
}
__device__ __noinline__ void wait_ge_shared_slow(volatile int* p, int target, long long spin, SyncWords* sync,
                                                 int64_t n) {
  const long long t0 = clock64();
  for (int k = 1;; ++k) {
    __nanosleep(32);
    if (*p >= target) return;
    if ((k & 63) == 0 && *(volatile unsigned int*)&sync->status != 0u) return;
    if (clock64() - t0 > spin) {
      latch_timeout(sync, n);
      return;
    }
  }
}
__device__ __forceinline__ void wait_ge_shared(volatile int* p, int target, long long spin, SyncWords* sync,
                                               int64_t n) {
  if (*p < target) wait_ge_shared_slow(p, target, spin, sync, n);
  __threadfence_block();
}

// ---------------------------------------------------------------- inner columns
// rows n0 .. n0+h-1, columns 0 .. D-1, row by row (every thread of the CTA)
__device__ __noinline__ void inner_rows(int64_t n0, int h) {
  const InstDesc& I = s_I;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int D = I.D;
  for (int r = 0; r < h; ++r) {
    const int64_t n = n0 + r;
    const int nslot = (int)(n % I.R);
    float2* row0 = I.ring + (int64_t)nslot * I.stride;
    const float2* lo_rd = I.lo_in + (int64_t)((n - 1) & 1) * I.dpad;
    float2* lo_wr = I.lo_in + (int64_t)(n & 1) * I.dpad;
    const float2 R2 = I.rowscal32[2 * n + 1];
    float2* snap = (I.tstep >= 0 && n % (I.tstep + 1) == 0) ? I.snaps + (n / (I.tstep + 1)) * I.nx : nullptr;
    float2 ycar = I.bnd32[2 * n];  // psi(-a, n delta): the value left of column 0
    float nacc = 0.f;
    for (int c0 = 0; c0 < D; c0 += kBand * kInnerPer) {
      const int cw = (D - c0 < kBand * kInnerPer) ? D - c0 : kBand * kInnerPer;
      const int L = (cw + kBand - 1) / kBand;
      const int j0 = c0 + tid * L;
      const int j1 = (j0 + L < c0 + cw) ? j0 + L : c0 + cw;
      // sources of the thread's columns, and its segment as an affine map y -> P y + Y
      float2 rv[kInnerPer], av[kInnerPer];
      float2 P = f2(1.f, 0.f), Y = f2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < kInnerPer; ++u) {
        rv[u] = av[u] = f2(0.f, 0.f);
        if (j0 + u < j1) {
          const int j = j0 + u;
          float2 ah, al;
          float2 S = rhs_inner32(I, n, nslot, j, R2, &ah);
          if (j == 0) {  // a = psi(-a, (n-1) delta), exact as hi + lo
            ah = I.bnd32[2 * (n - 1)];
            al = I.bnd32[2 * (n - 1) + 1];
          } else {
            al = lo_rd[j - 1];
          }
          S = add(S, al);
          rv[u] = S;
          av[u] = ah;
          Y = add(ah, fmac(I.c2lo, Y, fmac(I.c2, Y, S)));
          P = mulc(P, I.c2);
        }
      }
      // inclusive scan of the maps over the lanes: (earlier) then (later) =
      // (P_e P_l, P_l Y_e + Y_l)
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const float2 Pp = shfl_up2(P, off), Yp = shfl_up2(Y, off);
        if (lane >= off) {
          Y = fmac(Yp, P, Y);
          P = mulc(Pp, P);
        }
      }
      if (lane == 31) {
        s_scP[warp] = P;
        s_scY[warp] = Y;
      }
      float2 Pe = shfl_up2(P, 1), Ye = shfl_up2(Y, 1);
      if (lane == 0) {
        Pe = f2(1.f, 0.f);
        Ye = f2(0.f, 0.f);
      }
      __syncthreads();
      float2 Pw = f2(1.f, 0.f), Yw = f2(0.f, 0.f);
      for (int q = 0; q < warp; ++q) {
        const float2 Pq = s_scP[q], Yq = s_scY[q];
        Yw = fmac(Yw, Pq, Yq);
        Pw = mulc(Pw, Pq);
      }
      // the carry into the segment: the maps of every earlier segment applied to ycar
      float2 y = fmac(mulc(Pw, Pe), ycar, fmac(Yw, Pe, Ye));
#pragma unroll
      for (int u = 0; u < kInnerPer; ++u) {
        if (j0 + u < j1) {
          const int j = j0 + u;
          const float2 S = fmac(I.c2lo, y, fmac(I.c2, y, rv[u]));
          float2 sv, e;
          two_sum(av[u].x, S.x, sv.x, e.x);
          two_sum(av[u].y, S.y, sv.y, e.y);
          row0[j] = sv;
          lo_wr[j] = e;
          if (j == D - 1) I.lo_edge[n] = e;
          if (snap) snap[j] = sv;
          const float wt = (j == I.nx - 1) ? 0.5f : 1.0f;
          nacc = fmaf(wt * sv.x, sv.x, nacc);
          nacc = fmaf(wt * sv.y, sv.y, nacc);
          y = sv;
        }
      }
      if (j0 < j1 && j1 == c0 + cw) s_ylast = y;  // carry into the next pass
      __syncthreads();  // row n's inner columns are stored; the scan buffers are free
      ycar = s_ylast;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nacc += __shfl_down_sync(0xffffffffu, nacc, o);
    if (lane == 0) s_wn[warp][r] = nacc;
  }
}

// ---------------------------------------------------------------- sweep of x > a
// Lane l of a warp marches row n = nw + l (nw: the warp's first row) one column per
// step, one column behind lane l-1: at step k it takes column j = D + q, q = k - l.
// The warp's 32 rows at step k then share the anti-diagonal d = n + q = nw + k, so
// its stores and its reads of the delay row n-D (d - 2D) are 32 consecutive entries
// of the skew ring.

// a lane's prefetched operands of one step: the delay value (row n-D, column q) and
// the source tables at i = n-1-q (zero-padded: 0 out of the light cone)
struct Pre {
  float2 d, e, f;
};

// the constants of one lane's sweep (what only the edges use is read from I there)
struct SweepC {
  float2* skew;
  const float2* __restrict__ detab32;
  const float2* __restrict__ phitab32;
  int R, n, nslot, sD, lane, warp, D, nx, ncols, rd;
  bool row_on, useD, is_last, snap, hand_out;  // hand_out: lane 31 feeding the warp below
  float2 R1, R2, d1, c2, c3, d1l, c2l, c3l;  // c3, c3l: 0 for rows without the delay square (n <= D)
};
__device__ __forceinline__ float2* snap_row(const InstDesc& I, int n) {
  return I.snaps + (int64_t)(n / (I.tstep + 1)) * I.nx;
}

// its running state
struct SweepS {
  float2 y, a_hi, a_lo, o_hi, o_lo, o_hn, dprev;
  float nsum, ncomp;       // the row's norm so far: Kahan sum over its columns in order
  int dout;                // d-row (mod rd) of this step's outputs
  int dpre;                // d-row (mod rd) of the delay value kPre steps ahead
  Pre pq[kPre];
  // fast path (no wrap of the d-rows in the group): the same as pointers
  float2* pout;
  const float2* pdel;
  const float2* pe;
  const float2* pf;
};

__device__ __forceinline__ Pre sweep_fetch(const SweepC& c, int k, int dpre) {
  const int q = k - c.lane;
  Pre v;
  const float2 z = f2(0.f, 0.f);
  if (!c.useD) v.d = z;
  else if (q >= c.D) v.d = c.skew[(int64_t)dpre * c.R + c.sD];
  else v.d = (q >= 0) ? s_I.ring[(int64_t)c.sD * s_I.stride + q] : z;  // inner ring, row n-D
  const int i = c.n - 1 - q;
  v.e = c.detab32[i];
  v.f = c.phitab32[i - c.D];
  return v;
}

// the update of one column from S's parts: common to both steps
__device__ __forceinline__ void sweep_core(const SweepC& c, SweepS& st, float2 hn, float2 b_hi, float2 hp, float2 S,
                                           float2 L, float2& sv, float2& e) {
  // b (row n-1, column j) and the delay pair of row n-D-1 from the lane above, and
  // y (row n, column j-1), enter last: c2 (b + y) + c3 hp
  S = add(S, st.a_lo);
  const float2 t = add(b_hi, st.y);
  S = fmac(c.c2, t, S);
  S = fmac(c.c3, hp, S);
  L = fmac(c.c3l, hp, L);
  L = fmac(c.c2l, t, L);
  S = add(S, L);
  two_sum(st.a_hi.x, S.x, sv.x, e.x);
  two_sum(st.a_hi.y, S.y, sv.y, e.y);
}

__device__ __forceinline__ void norm_add(SweepS& st, float x) {  // Kahan
  const float yk = x - st.ncomp;
  const float tk = st.nsum + yk;
  st.ncomp = (tk - st.nsum) - yk;
  st.nsum = tk;
}

// a step where every lane marches a column of x > 3a (j >= 2D) other than the last,
// D >= 32 and no d-row wraps: operands by pointer, no tests
template <int QI>
__device__ __forceinline__ void sweep_step_fast(const SweepC& c, SweepS& st, int k, float2 b_hi, float2 b_lo,
                                                float2 hp) {
  const Pre pv = st.pq[QI];
  const float2 hn = add(st.dprev, pv.d);
  // the terms known before the lane above delivers row n-1: a (row n-1, column j-1),
  // the delay pair of row n-D, the sources, a's remainder
  float2 S = mulc(c.d1, st.a_hi);
  float2 L = mulc(c.d1l, st.a_hi);
  S = fmac(c.c3, hn, S);
  L = fmac(c.c3l, hn, L);
  S = fmac(c.R1, pv.e, S);
  S = fmac(c.R2, pv.f, S);
  float2 sv, e;
  sweep_core(c, st, hn, b_hi, hp, S, L, sv, e);
  *st.pout = sv;
  st.pout += c.R;
  const int q = k - c.lane;
  if (c.is_last) s_I.lo_row[c.D + q] = e;
  if (c.hand_out) s_queue[c.warp + 1][q & (kHandQ - 1)] = Hand{sv, e, hn};
  norm_add(st, fmaf(sv.x, sv.x, sv.y * sv.y));
  st.o_hi = sv;
  st.o_lo = e;
  st.o_hn = hn;
  st.y = sv;
  st.a_hi = b_hi;
  st.a_lo = b_lo;
  st.dprev = pv.d;
  // the operands kPre steps ahead
  Pre nv;
  nv.d = c.useD ? *st.pdel : f2(0.f, 0.f);
  nv.e = *st.pe;
  nv.f = *st.pf;
  st.pq[QI] = nv;
  st.pdel += c.R;
  --st.pe;
  --st.pf;
}

// any other step (pipeline edges, a < x <= 3a, the last column, D < 32, d-row wraps)
template <int QI>
__device__ __forceinline__ void sweep_step_gen(const SweepC& c, SweepS& st, int k, float2 b_hi, float2 b_lo, float2 hp) {
  const int q = k - c.lane;
  const bool act = c.row_on && (unsigned)q < (unsigned)c.ncols;
  const int j = c.D + q;
  const Pre pv = st.pq[QI];
  const float2 hn = add(st.dprev, pv.d);
  float2 S = mulc(c.d1, st.a_hi);
  float2 L = mulc(c.d1l, st.a_hi);
  S = fmac(c.c3, hn, S);
  L = fmac(c.c3l, hn, L);
  if (j >= 2 * c.D) {
    S = fmac(c.R1, pv.e, S);
    S = fmac(c.R2, pv.f, S);
  } else if (act) {
    S = general_extra32(c.n, c.nslot, j, c.R2, S);
  }
  float2 sv, e;
  sweep_core(c, st, hn, b_hi, hp, S, L, sv, e);
  if (act) {
    c.skew[(int64_t)st.dout * c.R + c.nslot] = sv;
    if (c.snap) snap_row(s_I, c.n)[j] = sv;
    if (c.is_last) s_I.lo_row[j] = e;
    if (c.hand_out) s_queue[c.warp + 1][q & (kHandQ - 1)] = Hand{sv, e, hn};
    const float wt = (j == c.nx - 1) ? 0.5f : 1.0f;
    norm_add(st, wt * fmaf(sv.x, sv.x, sv.y * sv.y));
    st.o_hi = sv;
    st.o_lo = e;
    st.o_hn = hn;
    st.y = sv;
    st.a_hi = b_hi;
    st.a_lo = b_lo;
    st.dprev = pv.d;
  }
  if (c.D < 32) __syncwarp();  // a lane may read the row of a lane D below soon
  st.dout = (st.dout + 1 == c.rd) ? 0 : st.dout + 1;
  st.pq[QI] = sweep_fetch(c, k + kPre, st.dpre);
  st.dpre = (st.dpre + 1 == c.rd) ? 0 : st.dpre + 1;
}

// the ring entry of row r (>= 0), column col (0 <= col < nx)
__device__ __forceinline__ const float2* ring_at(const InstDesc& I, int r, int col) {
  if (col < I.D) return I.ring + (int64_t)(r % I.R) * I.stride + col;
  return I.skew + (int64_t)((r + col - I.D) % (int)I.rd) * I.R + (r % I.R);
}

// warp 0: issue the cp.async copies of chunk ch of the previous band's last row np
// (value, remainder) and of its delay row np-D into buffer ch & 1, after waiting
// (bounded, when wait_prev) until that band has done the chunk after it
__device__ __noinline__ void stage_chunk(int ch, int np, int ncols, bool wait_prev, const unsigned long long* prev_word,
                                         unsigned long long tag_prev, SyncWords* sync) {
  const InstDesc& I = s_I;
  const int lane = threadIdx.x & 31, D = I.D;
  if (wait_prev && lane == 0) {
    const int cols = (ch + 1) * kChunk;
    wait_ge_global(prev_word, tag_prev + (unsigned long long)(cols < ncols ? cols : ncols), I.spin, sync, np + 1);
  }
  __syncwarp();
  const float2 z = f2(0.f, 0.f);
  const bool pd = (np >= D);
  const int b = ch & 1, q = ch * kChunk + lane;
  if (q < ncols) {
    cp_async8(&s_pv_hi[b][lane], ring_at(I, np, D + q));
    cp_async8(&s_pv_lo[b][lane], I.lo_row + D + q);
    if (pd) cp_async8(&s_pv_d[b][lane + 1], ring_at(I, np - D, q));
    else s_pv_d[b][lane + 1] = z;
  }
  if (lane == 0 && ch * kChunk < ncols) {  // the delay value left of the chunk's first column
    if (!pd) s_pv_d[b][0] = z;
    else if (ch == 0) s_pv_d[b][0] = psi_left32(I, np - D, -(D >> 1));
    else cp_async8(&s_pv_d[b][0], ring_at(I, np - D, ch * kChunk - 1));
  }
  cp_async_commit();
}

// warp 0: chunk ch (in shared memory) into its input queue, in the format of the
// queues between warps: entry q & 63 = (value, remainder, delay pair sum) of column q
__device__ __forceinline__ void chunk_to_queue(int ch) {
  const int lane = threadIdx.x & 31, b = ch & 1;
  s_queue[0][(ch * kChunk + lane) & (kHandQ - 1)] =
      Hand{s_pv_hi[b][lane], s_pv_lo[b][lane], add(s_pv_d[b][lane], s_pv_d[b][lane + 1])};
  __syncwarp();
}

// rows n0 .. n0+h-1 (row n0+tid on thread tid), columns D .. nx-1.  wait_prev:
// band c-1 (progress word prev_word, first row n0-256) is still being marched.
__device__ __noinline__ void sweep(int n0, int h, bool wait_prev, const unsigned long long* prev_word,
                                   unsigned long long* my_word, SyncWords* sync) {
  const InstDesc& I = s_I;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (warp * 32 >= h) return;
  const float2 z = f2(0.f, 0.f);
  const int D = I.D, Dh = D >> 1, R = I.R;
  const int nx = (int)I.nx, ncols = nx - D;
  const long long spin = I.spin;
  const bool row_on = tid < h;
  const int n = n0 + (row_on ? tid : 0);
  const int nw = n0 + 32 * warp;
  const bool next_on = (warp + 1 < kWarps) && ((warp + 1) * 32 < h);
  const bool warp_full = (warp + 1) * 32 <= h;
  const int t_last = h - 1;
  const bool is_last = (tid == t_last);
  const bool last_warp = (warp == (t_last >> 5));
  const unsigned long long tag = (unsigned long long)n0 << 32;
  auto inner_norm = [&]() {  // the row's inner columns (the inner pass's warp sums)
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += (double)s_wn[w][tid];
    return t;
  };
  if (ncols <= 0) {
    const double inner = row_on ? inner_norm() : 0.0;
    if (row_on) I.norms[n] = I.delta * (inner + I.bnorm[n]);
    if (last_warp) {
      __syncwarp();
      if (is_last) st_release_u64(my_word, tag);
    }
    return;
  }

  SweepC c;
  c.skew = I.skew;
  c.detab32 = I.detab32;
  c.phitab32 = I.phitab32;
  c.R = R;
  c.n = n;
  c.nslot = n % R;
  c.sD = (c.nslot >= D) ? c.nslot - D : c.nslot - D + R;
  c.lane = lane;
  c.D = D;
  c.nx = nx;
  c.ncols = ncols;
  c.rd = (int)I.rd;
  c.row_on = row_on;
  const bool hasD = row_on && n >= D;
  c.useD = hasD && D >= kPre;  // a delay value kPre steps ahead is not yet written when D < kPre
  const bool sqon = row_on && n >= D + 1;
  c.is_last = is_last;
  c.R1 = I.rowscal32[2 * n];
  c.R2 = I.rowscal32[2 * n + 1];
  c.snap = row_on && I.tstep >= 0 && n % (I.tstep + 1) == 0;
  c.warp = warp;
  c.hand_out = (lane == 31 && next_on);
  c.d1 = I.d1;
  c.c2 = I.c2;
  c.c3 = sqon ? I.c3 : z;
  c.d1l = I.d1lo;
  c.c2l = I.c2lo;
  c.c3l = sqon ? I.c3lo : z;
  const bool direct_d = hasD && D < kPre;
  // a warp holding a snapshot row takes the general step throughout
  const bool warp_snap = __any_sync(0xffffffffu, c.snap);

  // state at column D: y = psi[n][D-1] (inner pass), a = psi[n-1][D-1] + its remainder,
  // the delay value left of storage column 0 (x <= -a)
  SweepS st;
  const int s1 = (c.nslot >= 1) ? c.nslot - 1 : c.nslot - 1 + R;
  st.y = row_on ? I.ring[(int64_t)c.nslot * I.stride + D - 1] : z;
  st.a_hi = row_on ? I.ring[(int64_t)s1 * I.stride + D - 1] : z;
  st.a_lo = row_on ? I.lo_edge[n - 1] : z;
  st.dprev = hasD ? psi_left32(I, n - D, -Dh) : z;
  st.o_hi = st.o_lo = st.o_hn = z;
  st.nsum = 0.f;
  st.ncomp = 0.f;
  st.dout = ((nw % c.rd) + c.rd) % c.rd;
  st.dpre = (((nw - 2 * D) % c.rd) + c.rd) % c.rd;
#pragma unroll
  for (int u = 0; u < kPre; ++u) {
    st.pq[u] = sweep_fetch(c, u, st.dpre);
    st.dpre = (st.dpre + 1 == c.rd) ? 0 : st.dpre + 1;
  }

  // warp 0: the previous band's last row through shared memory, a chunk ahead
  if (warp == 0) {
    const unsigned long long tag_prev = (unsigned long long)(n0 - kBand) << 32;
    stage_chunk(0, n0 - 1, ncols, wait_prev, prev_word, tag_prev, sync);
    stage_chunk(1, n0 - 1, ncols, wait_prev, prev_word, tag_prev, sync);
    cp_async_wait1();  // chunk 0 is in shared memory
    __syncwarp();
    chunk_to_queue(0);
  }


  // steps [kfast0, kfast1): every lane marching a column j >= 2D other than the last
  const int kfast0 = D + 31, kfast1 = ncols - 1;
  const int kend = (ncols + 31 + kGrp - 1) / kGrp * kGrp;
  for (int kb = 0; kb < kend; kb += kGrp) {
    // ---- bookkeeping every kGrp steps
    __syncwarp();
    if (warp == 0 && kb > 0 && (kb % kChunk) == 0) {  // chunk ch+1 on its way, chunk ch in place
      stage_chunk(kb / kChunk + 1, n0 - 1, ncols, wait_prev, prev_word, (unsigned long long)(n0 - kBand) << 32, sync);
      cp_async_wait1();
      __syncwarp();
      chunk_to_queue(kb / kChunk);
    }
    if (last_warp && (kb % kChunk) == 0 && is_last) {  // progress of the band's last row, for band c+1
      const int done = kb - lane;
      st_release_u64(my_word, ((unsigned long long)n0 << 32) + (unsigned long long)(done < 0 ? 0 : (done > ncols ? ncols : done)));
    }
    if (warp > 0 && lane == 0) {  // consumer of the warp above
      __threadfence_block();
      ((volatile int*)s_cons)[warp] = (kb < ncols) ? kb : ncols;
      const int need = (kb + 2 * kGrp < ncols) ? kb + 2 * kGrp : ncols;
      wait_ge_shared((volatile int*)s_prod + warp - 1, need, spin, sync, n0);
    }
    if (next_on && lane == 31) {  // producer for the warp below
      __threadfence_block();
      const int done = kb - 31;
      ((volatile int*)s_prod)[warp] = (done < 0) ? 0 : (done > ncols ? ncols : done);
      const int need = kb + kGrp - 32 - kHandQ + 1;  // the entries this group overwrites were consumed
      if (need > 0) wait_ge_shared((volatile int*)s_cons + warp + 1, (need < ncols) ? need : ncols, spin, sync, n0);
    }
    __syncwarp();

    const bool fast = warp_full && !warp_snap && D >= 32 && kb >= kfast0 && kb + kGrp <= kfast1 &&
                      st.dout + kGrp < c.rd && st.dpre + kGrp < c.rd;
    if (fast) {
      st.pout = c.skew + (int64_t)st.dout * R + c.nslot;
      st.pdel = c.skew + (int64_t)st.dpre * R + c.sD;
      const int i = n - 1 - (kb + kPre - lane);  // the tables at step kb + kPre
      st.pe = c.detab32 + i;
      st.pf = c.phitab32 + (i - D);
      for (int uu = 0; uu < kGrp; uu += kPre) {
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
          const int k = kb + uu + u;
          // row n-1 at this step's column: from the lane above (its previous step), lane 0
          // from its queue (every lane reads the same entry: a broadcast, no branch)
          float2 b_hi = shfl_up2(st.o_hi, 1), b_lo = shfl_up2(st.o_lo, 1), hp = shfl_up2(st.o_hn, 1);
          const Hand hd = s_queue[warp][k & (kHandQ - 1)];
          if (lane == 0) {
            b_hi = hd.hi;
            b_lo = hd.lo;
            hp = hd.hn;
          }
          if (u == 0) sweep_step_fast<0>(c, st, k, b_hi, b_lo, hp);
          else sweep_step_fast<1>(c, st, k, b_hi, b_lo, hp);
        }
      }
      st.dout += kGrp;
      st.dpre += kGrp;
    } else {
      for (int uu = 0; uu < kGrp; uu += kPre) {
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
          const int k = kb + uu + u;
          float2 b_hi = shfl_up2(st.o_hi, 1), b_lo = shfl_up2(st.o_lo, 1), hp = shfl_up2(st.o_hn, 1);
          const Hand hd = s_queue[warp][k & (kHandQ - 1)];
          if (lane == 0) {  // (an entry past the last column is stale; lane 0 is idle then)
            b_hi = hd.hi;
            b_lo = hd.lo;
            hp = hd.hn;
          }
          if (direct_d) {  // D < kPre: the delay value is read at its step
            const int q = k - lane;
            st.pq[u].d = ((unsigned)q < (unsigned)ncols) ? *ring_at(I, n - D, q) : z;
          }
          if (u == 0) sweep_step_gen<0>(c, st, k, b_hi, b_lo, hp);
          else sweep_step_gen<1>(c, st, k, b_hi, b_lo, hp);
        }
      }
    }
  }
  __syncwarp();
  if (next_on && lane == 31) {
    __threadfence_block();
    ((volatile int*)s_prod)[warp] = ncols;
  }
  if (is_last) st_release_u64(my_word, ((unsigned long long)n0 << 32) + (unsigned long long)ncols);
  if (row_on) I.norms[n] = I.delta * (inner_norm() + ((double)st.nsum - (double)st.ncomp) + I.bnorm[n]);
}

// row r of an instance between its rings and a row-major buffer (see RowMap)
__global__ void k_row_move(RowMap m, int64_t r, float2* buf, int dir) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= m.nx) return;
  float2* e = (j < m.D) ? m.ring + (r % m.R) * m.stride + j
                        : m.skew + ((r + j - m.D) % m.rd) * (int64_t)m.R + (r % m.R);
  if (dir == 0) buf[j] = *e;
  else *e = (dir == 1) ? buf[j] : make_float2(0.f, 0.f);
}

cudaError_t launch_row_move(const RowMap& m, int64_t r, float2* buf, int dir, cudaStream_t s) {
  if (m.nx <= 0) return cudaSuccess;
  k_row_move<<<(unsigned)((m.nx + 255) / 256), 256, 0, s>>>(m, r, buf, dir);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kF32Threads, 2)
    k_march_f32c(const InstDesc* __restrict__ insts, const WorkItem* __restrict__ items, int nitems,
                 unsigned int* queue, SyncWords* sync) {

  const int tid = threadIdx.x;
  for (;;) {
    // the next band stream: bands stream, stream + g, ... of one instance
    if (tid == 0) {
      const unsigned q = atomicAdd(queue, 1u);
      s_item = (q < (unsigned)nitems) ? (int)q : -1;
    }
    __syncthreads();
    const int item = s_item;
    if (item < 0) break;
    const WorkItem Wk = items[item];
    {
      const int* src = reinterpret_cast<const int*>(&insts[Wk.inst]);
      int* dst = reinterpret_cast<int*>(&s_I);
      for (int k = tid; k < (int)(sizeof(InstDesc) / sizeof(int)); k += kF32Threads) dst[k] = src[k];
    }
    __syncthreads();
    if (s_I.range[0] < s_I.range[1]) {
      const InstDesc& I = s_I;
      const int g = Wk.g, r = Wk.stream;
      const int64_t nb = I.range[0], ne = I.range[1];
      unsigned long long* gdone = I.bsync;        // rows whose inner columns are complete
      unsigned long long* prog = I.bsync + 1;     // per stream: (first row of its band << 32) + columns
      for (int64_t n0 = nb + (int64_t)r * kBand; n0 < ne; n0 += (int64_t)g * kBand) {
        const int h = (int)((ne - n0 < kBand) ? ne - n0 : kBand);
        const bool first = (n0 == nb);
        if (tid == 0 && !first) wait_ge_global(gdone, (unsigned long long)n0, I.spin, sync, n0);
        __syncthreads();  // also: every warp has finished the previous band's sweep
        if (tid < kWarps) {
          s_prod[tid] = 0;
          s_cons[tid] = 0;
        }
        inner_rows(n0, h);
        __syncthreads();
        if (tid == 0) st_release_u64(gdone, (unsigned long long)(n0 + h));
        sweep((int)n0, h, !first && g > 1, prog + (r + g - 1) % g, prog + r, sync);
      }
    }
    __syncthreads();  // s_item and s_I are read by every thread before they are rewritten
  }
}

// FP32 copies of the boundary tables an instance's march reads, and the
// boundary column psi(-a, n delta) = C phi(-a - n delta) e(n delta) as an FP32
// hi/lo pair with its FP64 trapezoid end term delta-free (1/2)|psi|^2
__global__ void k_tables32(InstDesc I, const cd* detab, const cd* rowscal) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  auto cv = [](cd v) { return make_float2((float)v.re, (float)v.im); };
  if (i < I.nt) {
    const cd ex = I.C * (I.phitab[i] * I.etab[i]);
    const float2 hi = cv(ex);
    const_cast<float2*>(I.bnd32)[2 * i] = hi;
    const_cast<float2*>(I.bnd32)[2 * i + 1] = make_float2((float)(ex.re - (double)hi.x), (float)(ex.im - (double)hi.y));
    const_cast<double*>(I.bnorm)[i] = 0.5 * cabs2(ex);
    const_cast<float2*>(I.etab32)[i] = cv(I.etab[i]);
    const_cast<float2*>(I.rowscal32)[2 * i] = cv(rowscal[2 * i]);
    const_cast<float2*>(I.rowscal32)[2 * i + 1] = cv(rowscal[2 * i + 1]);
  }
  if (i < I.nphi) const_cast<float2*>(I.phitab32)[i] = cv(I.phitab[i]);
  if (i < I.nt + I.D) const_cast<float2*>(I.detab32)[i] = cv(detab[i]);
}

// advance every instance by `rows` rows: range = [done, min(done + rows, nt))
__global__ void k_advance(InstDesc* insts, int ninst, int64_t rows) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  int64_t done = insts[i].range[1];
  int64_t end = done + rows;
  if (end > insts[i].nt) end = insts[i].nt;
  insts[i].range[0] = done;
  insts[i].range[1] = end;
}

cudaError_t launch_tables32(const InstDesc& I, const cd* detab, const cd* rowscal, cudaStream_t s) {
  int64_t n = I.nphi > I.nt + I.D ? I.nphi : I.nt + I.D;
  k_tables32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(I, detab, rowscal);
  return cudaGetLastError();
}

cudaError_t launch_advance(InstDesc* insts, int ninst, int64_t rows, cudaStream_t s) {
  k_advance<<<(ninst + 127) / 128, 128, 0, s>>>(insts, ninst, rows);
  return cudaGetLastError();
}

int march_f32c_blocks_per_sm() {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march_f32c, kF32Threads, 0) != cudaSuccess) return 0;
  return per;
}

// every CTA resident (cooperative): a band stream may wait on a stream later in the
// queue only while fewer CTAs than its gang are busy, so grid >= the widest gang
// leaves no wait without a CTA to end it
cudaError_t launch_march_f32c(const InstDesc* insts, const WorkItem* items, int nitems, unsigned int* queue,
                              SyncWords* sync, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kF32Threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_march_f32c, insts, items, nitems, queue, sync);
}

}  // namespace fdtd
