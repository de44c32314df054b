// march_dw.cu -- the march of Eq. 1 in x > -a to FP64 accuracy in double-float
// arithmetic (pairs of FP32 numbers), for GPUs whose FP64 rate is a small
// fraction of their FP32 rate.
//
// The update is the one of march_f64.cu (Eq. 3a-c squares for line 1 with the
// delay term as App. A writes it, Eq. 4 bars for lines 2-3, line 4 at the
// square centre):
//   psi[n][m] = c1 psi[n-1][m-1] + c2 (psi[n-1][m] + psi[n][m-1])
//             + c3 [n >= D+1] (delay square) + (1/A)(S2 + S3 + Schi).
// Every value is a double-float: x = x_h + x_l, two FP32 numbers with
// |x_l| <= ulp(x_h)/2, 48 significant bits.  Sums use Knuth's TwoSum, products
// Dekker's product through an FMA (the rounding error of x_h y_h is exact), and
// the cross terms x_h y_l + x_l y_h enter the low word; the x_l y_l term, below
// 2^-48 of the product, is dropped.  Written as
//   psi[n][m] = a + S + c2 psi[n][m-1],   a = psi[n-1][m-1],   c1 = 1 + d1,
// the only term with weight ~1 is a, which is carried exactly; S is
// O(|W delta|) |psi| and the row recurrence y_m = c2 y_{m-1} + r_m is the same
// as in FP64.  The boundary tables are FP64 tables split into double-floats
// once per boundary; the per-CTA norm partials are reduced in FP64.
//
// Work layout: persistent cooperative CTAs, two per SM (while one waits at a
// barrier or on a neighbour, the other computes); CTA b owns the columns
// [colsplit[b], colsplit[b+1]) of every row, each thread a contiguous segment
// of them, with the recurrence carried across segments and CTAs as in
// march_f64.cu (a carry's influence dies as |c2|^k; it is carried exactly
// while that exceeds 2^-52, below double-float rounding).  Rows are not
// separated by a grid barrier.  Row n of CTA b needs, of each CTA it reads,
// only rows up to n - lag (lag 1 for the stencil and the carry halo from the
// CTA on its left, lag D for the delay term, lag 1 + j or j - D + 1 for the
// mirror bars of lines 2-3 in -a < x <= 3a, which read marched columns of
// earlier rows, some of them to the right).  Each CTA publishes the number of
// rows it has completed (a release store); before row n it waits (acquire
// loads, bounded) until every CTA it reads has completed the rows it needs,
// and until every CTA that reads it has gone far enough that the ring slot of
// row n is free: the ring holds D + 2 + kRowSlack rows, so a CTA may run up to
// kRowSlack rows ahead of its readers (RowDeps in fdtd_internal.cuh).  Every wait is for a strictly earlier
// row, so the order of rows is a well-founded order and no set of waits can
// close a cycle; co-residency of all CTAs (cooperative launch) does the rest.
// CTAs therefore run skewed, each a fraction of a row behind the CTA on its
// left, and the cost of a row barrier disappears.
//
// Reads of x <= -a use psi(x,t) = C phi(x-t) e(t) from the tables; beyond
// x > 3a the sources collapse to R1(n) [E(r2) - E(r2+D)] + R2(n) phi(r2).
#include <cuda_runtime.h>

#include "fdtd_internal.cuh"

namespace fdtd {

// ---------------------------------------------------------------- double-float
struct zc {
  float rh, ih, rl, il;  // (rh + rl) + i (ih + il)
};

__device__ __forceinline__ zc zc0() { return zc{0.f, 0.f, 0.f, 0.f}; }
__device__ __forceinline__ zc ldz(const float4* p) {
  const float4 v = *p;
  return zc{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ zc ldz_ro(const float4* p) {
  const float4 v = __ldg(p);
  return zc{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ void stz(float4* p, zc v) { *p = make_float4(v.rh, v.ih, v.rl, v.il); }
__device__ __forceinline__ zc zc_of(float4 v) { return zc{v.x, v.y, v.z, v.w}; }

// s + e = a + b exactly (Knuth); no contraction into FMAs
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (or a = 0); renormalises a pair
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// acc (unnormalised) += x * y, complex double-float
__device__ __forceinline__ void cmac(zc& a, const zc& x, const zc& y) {
  float p, e, s, t;
  // real part: x.r y.r - x.i y.i
  p = __fmul_rn(x.rh, y.rh);
  e = __fmaf_rn(x.rh, y.rh, -p);
  two_sum(a.rh, p, s, t);
  a.rh = s;
  float lr = __fadd_rn(a.rl, __fadd_rn(t, e));
  p = __fmul_rn(-x.ih, y.ih);
  e = __fmaf_rn(-x.ih, y.ih, -p);
  two_sum(a.rh, p, s, t);
  a.rh = s;
  lr = __fadd_rn(lr, __fadd_rn(t, e));
  lr = __fmaf_rn(x.rh, y.rl, lr);
  lr = __fmaf_rn(x.rl, y.rh, lr);
  lr = __fmaf_rn(-x.ih, y.il, lr);
  lr = __fmaf_rn(-x.il, y.ih, lr);
  a.rl = lr;
  // imaginary part: x.r y.i + x.i y.r
  p = __fmul_rn(x.rh, y.ih);
  e = __fmaf_rn(x.rh, y.ih, -p);
  two_sum(a.ih, p, s, t);
  a.ih = s;
  float li = __fadd_rn(a.il, __fadd_rn(t, e));
  p = __fmul_rn(x.ih, y.rh);
  e = __fmaf_rn(x.ih, y.rh, -p);
  two_sum(a.ih, p, s, t);
  a.ih = s;
  li = __fadd_rn(li, __fadd_rn(t, e));
  li = __fmaf_rn(x.rh, y.il, li);
  li = __fmaf_rn(x.rl, y.ih, li);
  li = __fmaf_rn(x.ih, y.rl, li);
  li = __fmaf_rn(x.il, y.rh, li);
  a.il = li;
}
// x * y into a fresh accumulator
__device__ __forceinline__ zc cmul(const zc& x, const zc& y) {
  zc a;
  float p, e, s, t;
  a.rh = __fmul_rn(x.rh, y.rh);
  float lr = __fmaf_rn(x.rh, y.rh, -a.rh);
  p = __fmul_rn(-x.ih, y.ih);
  e = __fmaf_rn(-x.ih, y.ih, -p);
  two_sum(a.rh, p, s, t);
  a.rh = s;
  lr = __fadd_rn(lr, __fadd_rn(t, e));
  lr = __fmaf_rn(x.rh, y.rl, lr);
  lr = __fmaf_rn(x.rl, y.rh, lr);
  lr = __fmaf_rn(-x.ih, y.il, lr);
  lr = __fmaf_rn(-x.il, y.ih, lr);
  a.rl = lr;
  a.ih = __fmul_rn(x.rh, y.ih);
  float li = __fmaf_rn(x.rh, y.ih, -a.ih);
  p = __fmul_rn(x.ih, y.rh);
  e = __fmaf_rn(x.ih, y.rh, -p);
  two_sum(a.ih, p, s, t);
  a.ih = s;
  li = __fadd_rn(li, __fadd_rn(t, e));
  li = __fmaf_rn(x.rh, y.il, li);
  li = __fmaf_rn(x.rl, y.ih, li);
  li = __fmaf_rn(x.ih, y.rl, li);
  li = __fmaf_rn(x.il, y.rh, li);
  a.il = li;
  return a;
}
// a + b (unnormalised)
__device__ __forceinline__ zc cadd(const zc& a, const zc& b) {
  zc r;
  float t;
  two_sum(a.rh, b.rh, r.rh, t);
  r.rl = __fadd_rn(t, __fadd_rn(a.rl, b.rl));
  two_sum(a.ih, b.ih, r.ih, t);
  r.il = __fadd_rn(t, __fadd_rn(a.il, b.il));
  return r;
}
// a - b (unnormalised)
__device__ __forceinline__ zc csub(const zc& a, const zc& b) {
  return cadd(a, zc{-b.rh, -b.ih, -b.rl, -b.il});
}
__device__ __forceinline__ zc cscale(float w, const zc& a) {  // w a power of two
  return zc{w * a.rh, w * a.ih, w * a.rl, w * a.il};
}
__device__ __forceinline__ zc cnorm(const zc& a) {
  zc r;
  fast_two_sum(a.rh, a.rl, r.rh, r.rl);
  fast_two_sum(a.ih, a.il, r.ih, r.il);
  return r;
}
// |y|^2 added to a real double-float accumulator (h, l), unnormalised
__device__ __forceinline__ void nacc_add(float& h, float& l, const zc& y) {
  float p, e, s, t;
  p = __fmul_rn(y.rh, y.rh);
  e = __fmaf_rn(y.rh, y.rh, -p);
  e = __fmaf_rn(y.rh + y.rh, y.rl, e);
  float q = __fmul_rn(y.ih, y.ih);
  float f = __fmaf_rn(y.ih, y.ih, -q);
  f = __fmaf_rn(y.ih + y.ih, y.il, f);
  two_sum(h, p, s, t);
  h = s;
  l = __fadd_rn(l, __fadd_rn(t, e));
  two_sum(h, q, s, t);
  h = s;
  l = __fadd_rn(l, __fadd_rn(t, f));
}

// ---------------------------------------------------------------- reads
// psi at x = c delta <= -a, t = r delta: phi((c-r) delta) C e(r delta)
__device__ __forceinline__ zc psi_left_dw(const DwArgs& A, int64_t r, int64_t c) {
  const int Dh = A.D >> 1;
  zc v = cmul(ldz_ro(&A.phitab[r - c - Dh]), ldz_ro(&A.etabC[r]));
  if (A.phitab2) cmac(v, ldz_ro(&A.phitab2[r - c - Dh]), ldz_ro(&A.etabC2[r]));  // second photon of a pair
  return cnorm(v);
}

// psi at an earlier point the update of row n reads; nslot = n % R
__device__ __forceinline__ zc psi_any_dw(const DwArgs& A, int64_t n, int nslot, int64_t r, int64_t c) {
  const int Dh = A.D >> 1;
  if (c <= -Dh) return psi_left_dw(A, r, c);
  int slot = nslot - (int)(n - r);
  if (slot < 0) slot += A.R;
  return ldz(&A.ring[(int64_t)slot * A.stride + (c + Dh - 1)]);
}

// r_m for a column of -a < x <= 3a: every term through psi_any_dw
__device__ __noinline__ zc rhs_general_dw(const DwArgs& A, int64_t n, int nslot, int64_t j, zc R2) {
  const int D = A.D, Dh = D >> 1;
  const int64_t m = j - Dh + 1;
  const zc a = psi_any_dw(A, n, nslot, n - 1, m - 1);
  zc S = cmul(zc_of(A.d1), a);
  cmac(S, zc_of(A.c2), psi_any_dw(A, n, nslot, n - 1, m));
  if (n >= D + 1) {
    const zc sq = cadd(cadd(psi_any_dw(A, n, nslot, n - D, m - D), psi_any_dw(A, n, nslot, n - D, m - D - 1)),
                       cadd(psi_any_dw(A, n, nslot, n - D - 1, m - D), psi_any_dw(A, n, nslot, n - D - 1, m - D - 1)));
    cmac(S, zc_of(A.c3), sq);
  }
  const int64_t r2 = n - m - Dh;  // line 2: t - x - a at the centre
  if (r2 >= 0) {
    const float w = (r2 == 0) ? 0.5f : 1.0f;
    const zc bl = cadd(psi_any_dw(A, n, nslot, r2, -m - D), psi_any_dw(A, n, nslot, r2, -m - D + 1));
    const zc br = cadd(psi_any_dw(A, n, nslot, r2, -m), psi_any_dw(A, n, nslot, r2, -m + 1));
    cmac(S, zc_of(A.gs), cscale(w, csub(bl, br)));
    cmac(S, R2, ldz_ro(&A.phitab[r2]));  // line 4: phi((m-n) delta) = phitab[r2]
    if (A.phitab2) cmac(S, ldz_ro(&A.rowscal2[2 * n + 1]), ldz_ro(&A.phitab2[r2]));
  }
  if (m >= Dh + 1) {  // line 3, theta(x - a)
    const int64_t r3 = n - m + Dh;
    if (r3 >= 0) {
      const float w = (r3 == 0) ? 0.5f : 1.0f;
      const zc bl = cadd(psi_any_dw(A, n, nslot, r3, D - m), psi_any_dw(A, n, nslot, r3, D - m + 1));
      const zc br = cadd(psi_any_dw(A, n, nslot, r3, -m), psi_any_dw(A, n, nslot, r3, -m + 1));
      cmac(S, zc_of(A.gs), cscale(w, csub(bl, br)));
    }
  }
  return cadd(a, S);
}

struct RowDw {
  int64_t n;
  int nslot;
  const float4* row1;
  const float4* rowD;
  const float4* rowD1;
  float4* row0;
  double2* snap;
  zc R1, R2;
  zc R1b, R2b;  // second term of a photon pair
  float4* hs;
  int64_t hbase;
  bool cold;
};

// r_m for x > 3a (j >= 2D): a + d1 a + c2 b + c3 (delay square) + R1 dE + R2 phi
__device__ __forceinline__ zc rhs_bulk_dw(const DwArgs& A, const RowDw& R, int64_t j) {
  const int D = A.D;
  const zc a = ldz(R.row1 + j - 1);
  const zc b = ldz(R.row1 + j);
  zc S = cmul(zc_of(A.d1), a);
  cmac(S, zc_of(A.c2), b);
  if (R.rowD) {
    const zc hn = cadd(ldz(R.rowD + j - D - 1), ldz(R.rowD + j - D));  // row n-D pair
    if (R.rowD1) {
      zc hp;
      if (R.hs && !R.cold) hp = zc_of(R.hs[j - R.hbase]);
      else hp = cadd(ldz(R.rowD1 + j - D - 1), ldz(R.rowD1 + j - D));
      cmac(S, zc_of(A.c3), cadd(hn, hp));
    }
    if (R.hs) R.hs[j - R.hbase] = make_float4(hn.rh, hn.ih, hn.rl, hn.il);
  }
  const int64_t i = R.n - j - 1 + D;  // r2 + D
  if (i >= 0) {
    cmac(S, R.R1, ldz_ro(&A.detab[i]));
    if (i >= D) cmac(S, R.R2, ldz_ro(&A.phitab[i - D]));
    if (A.detab2) {
      cmac(S, R.R1b, ldz_ro(&A.detab2[i]));
      if (i >= D) cmac(S, R.R2b, ldz_ro(&A.phitab2[i - D]));
    }
  }
  return cadd(a, S);
}

__device__ __forceinline__ zc rhs_dw(const DwArgs& A, const RowDw& R, int64_t j) {
  if (j >= 2 * (int64_t)A.D) return rhs_bulk_dw(A, R, j);
  return rhs_general_dw(A, R.n, R.nslot, j, R.R2);
}

// one step of the row recurrence: y_j = c2 y_{j-1} + r_j, normalised
__device__ __forceinline__ zc step_dw(const DwArgs& A, zc r, const zc& y) {
  cmac(r, zc_of(A.c2), y);
  return cnorm(r);
}
// the same with r_j's c2 b_j term still out: y_j = c2 (b_j + y_{j-1}) + r'_j (one product)
__device__ __forceinline__ zc step_b_dw(const DwArgs& A, zc r, const zc& b, const zc& y) {
  cmac(r, zc_of(A.c2), cadd(b, y));
  return cnorm(r);
}

__device__ __forceinline__ void finalize_dw(const DwArgs& A, const RowDw& R, int64_t j, const zc& y, float& nh,
                                            float& nl) {
  stz(R.row0 + j, y);
  if (R.snap) R.snap[j] = make_double2((double)y.rh + (double)y.rl, (double)y.ih + (double)y.il);
  nacc_add(nh, nl, y);  // the last column's half weight is taken off once per row
}

__global__ void __launch_bounds__(kDwThreads, kDwCtasPerSm) k_march_dw(const DwArgs A) {
  constexpr int P = kDwP;
  extern __shared__ float4 s_h[];  // pair sums, khalo + CTA range entries
  __shared__ zc s_last[kDwThreads];
  __shared__ int s_len[kDwThreads];
  __shared__ zc s_carry;
  __shared__ zc s_halo[kMaxTrunc];
  __shared__ float2 s_red[kDwThreads / 32];
  __shared__ double s_tot;
  __shared__ int s_ok;

  const int tid = threadIdx.x, cta = blockIdx.x;
  const int D = A.D, Dh = D >> 1;
  const int64_t j_lo = A.colsplit[cta], j_hi = A.colsplit[cta + 1];
  // segments as in march_f64.cu: equal odd lengths in x > 3a, cost-weighted otherwise
  const int64_t G2 = (2 * (int64_t)D < A.nx) ? 2 * (int64_t)D : A.nx;
  int64_t s0, s1;
  if (j_lo >= G2) {
    // odd lengths (the pair sums in shared memory stay free of bank conflicts); warp 0,
    // which also waits on the neighbours and forms the halo carry, takes 2 columns fewer
    const int64_t len = j_hi - j_lo;
    int64_t seg = ((len + 64 + kDwThreads - 1) / kDwThreads) | 1;
    if (seg < 3) seg = 3;
    const int64_t seg0 = seg - 2;
    s0 = (tid < 32) ? j_lo + (int64_t)tid * seg0 : j_lo + 32 * seg0 + (int64_t)(tid - 32) * seg;
    if (s0 > j_hi) s0 = j_hi;
    const int64_t sl = (tid < 32) ? seg0 : seg;
    s1 = (s0 + sl < j_hi) ? s0 + sl : j_hi;
  } else {
    const int64_t wm = A.mid_weight;
    auto cumw = [&](int64_t j) { return j <= G2 ? wm * j : wm * G2 + (j - G2); };
    auto inv = [&](int64_t x) { return x <= wm * G2 ? (x + wm - 1) / wm : G2 + (x - wm * G2); };
    const int64_t W0 = cumw(j_lo), W1 = cumw(j_hi);
    s0 = inv(W0 + (W1 - W0) * tid / kDwThreads);
    s1 = inv(W0 + (W1 - W0) * (tid + 1) / kDwThreads);
  }
  const int64_t h0 = (j_lo - A.khalo > 0) ? j_lo - A.khalo : 0;
  const int nh = (int)(j_lo - h0);
  s_len[tid] = (int)(s1 - s0);
  if (tid == 0) s_ok = (*(volatile unsigned int*)&A.sync->status == 0u) ? 1 : 0;
  __syncthreads();
  if (!s_ok) return;

  int slot = (int)(A.n_begin % A.R);  // ring slot of row n
  int64_t snap_ctr = -1, snap_idx = 0;  // row n is a snapshot row when snap_ctr == 0
  if (A.snaps && A.tstep >= 0) {
    snap_ctr = A.n_begin % (A.tstep + 1);
    snap_idx = A.n_begin / (A.tstep + 1) + (snap_ctr ? 1 : 0);
  }
  for (int64_t n = A.n_begin; n < A.n_end; ++n,
               slot = (slot + 1 == A.R) ? 0 : slot + 1,
               snap_idx += (snap_ctr == 0) ? 1 : 0,
               snap_ctr = (snap_ctr < 0) ? -1 : (snap_ctr == A.tstep ? 0 : snap_ctr + 1)) {
    // wait: the rows this CTA reads are complete, and its readers are past the
    // rows that the slot of row n still holds for them (warp 0, one flag per lane)
    if (tid < 32) {
      const bool ok = row_wait_warp(A.deps, A.sync, A.spin_cycles, A.n_begin, cta, n, kRowSlack);
      if (tid == 0) s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok) return;

    RowDw R;
    R.n = n;
    // ring slots and the snapshot row from running counters (no 64-bit division per row)
    auto back = [&](int k) { const int t = slot - k; return t < 0 ? t + A.R : t; };
    R.nslot = slot;
    R.row1 = A.ring + (int64_t)back(1) * A.stride;
    R.rowD = (n >= D) ? A.ring + (int64_t)back(D) * A.stride : nullptr;
    R.rowD1 = (n >= D + 1) ? A.ring + (int64_t)back(D + 1) * A.stride : nullptr;
    R.row0 = A.ring + (int64_t)slot * A.stride;
    R.snap = (snap_ctr == 0) ? A.snaps + snap_idx * A.nx : nullptr;
    R.R1 = ldz_ro(&A.rowscal[2 * n]);
    R.R2 = ldz_ro(&A.rowscal[2 * n + 1]);
    R.R1b = A.rowscal2 ? ldz_ro(&A.rowscal2[2 * n]) : zc0();
    R.R2b = A.rowscal2 ? ldz_ro(&A.rowscal2[2 * n + 1]) : zc0();
    R.hs = A.hreuse ? s_h : nullptr;
    R.hbase = h0;
    R.cold = (n == A.n_begin);

    // carry into column j_lo: the true psi[n][j_lo - 1], the recurrence over the
    // nh halo columns unrolled into a weighted sum (warp 0, one column per lane):
    //   y = sum_c c2^(nh-1-c) r_c  +  c2^nh psi(-a, t) [first CTA only]
    if (tid < 32 && j_lo < j_hi) {
      zc acc = zc0();
      for (int c = tid; c < nh; c += 32) cmac(acc, zc_of(A.c2pow[nh - 1 - c]), rhs_dw(A, R, h0 + c));
      if (tid == 0 && h0 == 0) cmac(acc, zc_of(A.c2pow[nh]), psi_left_dw(A, n, -Dh));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const zc other = zc{__shfl_down_sync(0xffffffffu, acc.rh, o), __shfl_down_sync(0xffffffffu, acc.ih, o),
                            __shfl_down_sync(0xffffffffu, acc.rl, o), __shfl_down_sync(0xffffffffu, acc.il, o)};
        acc = cadd(acc, other);
      }
      if (tid == 0) s_carry = cnorm(acc);
    }

    // pass A: the segment from a zero carry
    float nh_ = 0.f, nl_ = 0.f;
    zc y0[P];
    zc y = zc0();
    if (s0 >= 2 * (int64_t)D && s0 < s1 && !A.detab2) {
      // a segment of x > 3a only: each column's loads are issued one column ahead,
      // and the stencil and delay neighbours are carried from the column before
      // per-thread bases; column s0 + k is offset k (32-bit) from each
      const bool dd = R.rowD != nullptr, dd1 = R.rowD1 != nullptr;
      const bool use_hs = R.hs && !R.cold;
      const float4* b1 = R.row1 + s0;                     // row n-1 at column s0
      const float4* bD = dd ? R.rowD + (s0 - D) : b1;     // row n-D at column s0 - D
      const float4* bD1 = dd1 ? R.rowD1 + (s0 - D) : b1;  // row n-D-1 at column s0 - D
      float4* bh = R.hs ? R.hs + (s0 - R.hbase) : nullptr;
      const int64_t i0 = R.n - s0 - 1 + D;  // detab index of column s0 (r2 + D); one less per column
      // sources of column s0 + k: detab[i0 - k] while k <= kE, phitab[i0 - D - k] while k <= kF
      const int kE = (int)(i0 < 0 ? -1 : (i0 < (int64_t)(s1 - s0) ? i0 : s1 - s0));
      const int kF = (int)(i0 - D < 0 ? -1 : (i0 - D < (int64_t)(s1 - s0) ? i0 - D : s1 - s0));
      const float4* bE = A.detab + (i0 >= 0 ? i0 : 0);
      const float4* bF = A.phitab + (i0 - D >= 0 ? i0 - D : 0);
      const int len = (int)(s1 - s0);
      zc a = ldz(b1 - 1);
      zc pDp = dd ? ldz(bD - 1) : zc0();
      zc pD1p = (dd1 && !use_hs) ? ldz(bD1 - 1) : zc0();
      zc b_n = ldz(b1);
      zc pD_n = dd ? ldz(bD) : zc0();
      zc pD1_n = (dd1 && !use_hs) ? ldz(bD1) : zc0();
      zc hp_n = use_hs ? zc_of(bh[0]) : zc0();
      zc E_n = (kE >= 0) ? ldz_ro(bE) : zc0();
      zc F_n = (kF >= 0) ? ldz_ro(bF) : zc0();
      zc bcur = zc0();  // b of the column col() formed last
      auto col = [&](int k) -> zc {  // r' of column s0 + k (no c2 b) from the values loaded for it; loads for k + 1
        const zc b = b_n, pD = pD_n, pD1 = pD1_n, hpv = hp_n, E = E_n, Fv = F_n;
        const int k1 = k + 1;
        if (k1 < len) {
          b_n = ldz(b1 + k1);
          if (dd) pD_n = ldz(bD + k1);
          if (dd1 && !use_hs) pD1_n = ldz(bD1 + k1);
          if (use_hs) hp_n = zc_of(bh[k1]);
          E_n = (k1 <= kE) ? ldz_ro(bE - k1) : zc0();
          F_n = (k1 <= kF) ? ldz_ro(bF - k1) : zc0();
        }
        zc S = cmul(zc_of(A.d1), a);  // c2 b enters with c2 y in the step: c2 (b + y)
        if (dd) {
          const zc hn = cadd(pDp, pD);  // row n-D pair
          if (dd1) cmac(S, zc_of(A.c3), cadd(hn, use_hs ? hpv : cadd(pD1p, pD1)));
          if (bh) bh[k] = make_float4(hn.rh, hn.ih, hn.rl, hn.il);
        }
        if (k <= kE) {
          cmac(S, R.R1, E);
          if (k <= kF) cmac(S, R.R2, Fv);
        }
        const zc r = cadd(a, S);
        bcur = b;
        a = b;
        pDp = pD;
        pD1p = pD1;
        return r;
      };
#pragma unroll
      for (int v = 0; v < P; ++v) {
        if (v < len) {
          const zc r = col(v);
          y = step_b_dw(A, r, bcur, y);
        }
        y0[v] = y;
      }
      float4* o = R.row0 + s0;
      for (int k = P; k < len; ++k) {
        const zc r = col(k);
        y = step_b_dw(A, r, bcur, y);
        if (k < A.kfix) stz(o + k, y);  // provisional: receives the carry in pass B
        else finalize_dw(A, R, s0 + k, y, nh_, nl_);
      }
    } else {
#pragma unroll
      for (int v = 0; v < P; ++v) {
        const int64_t j = s0 + v;
        if (j < s1) y = step_dw(A, rhs_dw(A, R, j), y);
        y0[v] = y;
      }
      for (int64_t j = s0 + P; j < s1; ++j) {
        y = step_dw(A, rhs_dw(A, R, j), y);
        if (j - s0 < A.kfix) stz(R.row0 + j, y);  // provisional: receives the carry in pass B
        else finalize_dw(A, R, j, y, nh_, nl_);
      }
    }
    s_last[tid] = (s0 < s1) ? y : zc0();
    __syncthreads();

    // pass B: the carry from the threads before, added to the first kfix columns
    if (s0 < s1) {
      zc carry = zc0(), ap = zc{1.f, 0.f, 0.f, 0.f};
      for (int s = 1; s <= tid + 1; ++s) {
        if (tid - s >= 0) {
          cmac(carry, ap, s_last[tid - s]);
          const int lu = s_len[tid - s];
          ap = cnorm(cmul(ap, (lu <= kMaxTrunc) ? zc_of(A.c2pow[lu]) : zc0()));
          if (ap.rh * ap.rh + ap.ih * ap.ih < 5.0e-32f) break;  // (2^-52)^2
        } else {
          cmac(carry, ap, s_carry);
        }
      }
      carry = cnorm(carry);
#pragma unroll
      for (int v = 0; v < P; ++v) {
        const int64_t j = s0 + v;
        if (j < s1) {
          zc yv = y0[v];
          if (v < A.kfix) {
            cmac(yv, zc_of(A.c2pow[v + 1]), carry);
            yv = cnorm(yv);
          }
          finalize_dw(A, R, j, yv, nh_, nl_);
        }
      }
      for (int v = P; v < A.kfix && s0 + v < s1; ++v) {
        const int64_t j = s0 + v;
        zc yv = ldz(R.row0 + j);
        cmac(yv, zc_of(A.c2pow[v + 1]), carry);
        finalize_dw(A, R, j, cnorm(yv), nh_, nl_);
      }
    }

    // norm partial of this CTA: double-float across threads and warps (fixed order),
    // one conversion to FP64 per CTA and row
    {
      float h = nh_, l = nl_;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, h, o), l2 = __shfl_down_sync(0xffffffffu, l, o);
        float sv, t;
        two_sum(h, h2, sv, t);
        l = __fadd_rn(l, __fadd_rn(l2, t));
        h = sv;
      }
      if ((tid & 31) == 0) s_red[tid >> 5] = make_float2(h, l);
    }
    __syncthreads();  // every store of row n is issued
    // probes of row n in this CTA's columns
    if (A.probe_off && tid >= 32 && tid < 64) {
      const int k1 = A.probe_off[n + 1];
      for (int k = A.probe_off[n] + tid - 32; k < k1; k += 32) {
        const int j = A.probe_col[k];
        if (j >= j_lo && j < j_hi) {
          const float4 v = R.row0[j];
          A.probe_val[A.probe_idx[k]] = make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
        }
      }
    }
    if (tid < 32) {  // warp 0 sums the warps' partials
      constexpr int nw = kDwThreads / 32;
      float2 v = (tid < nw) ? s_red[tid] : make_float2(0.f, 0.f);
      float h = v.x, l = v.y;
#pragma unroll
      for (int o = nw / 2; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, h, o), l2 = __shfl_down_sync(0xffffffffu, l, o);
        float sv, t;
        two_sum(h, h2, sv, t);
        l = __fadd_rn(l, __fadd_rn(l2, t));
        h = sv;
      }
      if (tid == 0) s_tot = (double)h + (double)l;
    }
    if (tid == 0) {
      double tot = s_tot;
      if (j_hi == A.nx && j_lo < j_hi) {  // trapezoid end weight: half of the last column
        const float4 v = R.row0[A.nx - 1];
        const double re = (double)v.x + (double)v.z, im = (double)v.y + (double)v.w;
        tot -= 0.5 * (re * re + im * im);
      }
      A.partials[(n - A.n_begin) * gridDim.x + cta] = tot;
      if (!A.probe_off) {
        __threadfence();
        st_release_u64(&A.deps.done[cta], (unsigned long long)(n + 1));
      }
    }
    if (A.probe_off) {  // the probe values are written before the row is published
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release_u64(&A.deps.done[cta], (unsigned long long)(n + 1));
      }
    }
  }
}

// N(n) = delta [ (1/2)|psi(-a, n delta)|^2 + sum over CTAs of the partials ], FP64, fixed order
__global__ void k_norms_rows(const double* __restrict__ partials, int grid, int64_t n_begin, int64_t n_end,
                             const cd* __restrict__ etab, const cd* __restrict__ phitab,
                             const cd* __restrict__ etab2, const cd* __restrict__ phitab2, double C, double delta,
                             double* __restrict__ norms) {
  const int64_t n = n_begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= n_end) return;
  cd v = phitab[n] * etab[n];  // psi(-a, n delta) = C phi(-a - n delta) e(n delta): phitab[n]
  if (phitab2) v = v + phitab2[n] * etab2[n];
  v = C * v;
  double t = 0.5 * cabs2(v);
  const double* p = partials + (n - n_begin) * grid;
  for (int b = 0; b < grid; ++b) t += p[b];
  norms[n] = delta * t;
}

// split FP64 tables into double-floats; etabC = C e
__device__ __forceinline__ float4 split_dw(cd v) {
  const float rh = (float)v.re, ih = (float)v.im;
  return make_float4(rh, ih, (float)(v.re - (double)rh), (float)(v.im - (double)ih));
}
__global__ void k_tables_dw(const cd* etab, const cd* phitab, const cd* rowscal, const cd* detab, double C, int64_t nt,
                            int64_t nphi, int D, float4* etabC, float4* phi_dw, float4* rowscal_dw, float4* detab_dw) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nt) {
    etabC[i] = split_dw(C * etab[i]);
    rowscal_dw[2 * i] = split_dw(rowscal[2 * i]);
    rowscal_dw[2 * i + 1] = split_dw(rowscal[2 * i + 1]);
  }
  if (i < nphi) phi_dw[i] = split_dw(phitab[i]);
  if (i < nt + D) detab_dw[i] = split_dw(detab[i]);
}

__global__ void k_row_dw(const float4* __restrict__ src, int64_t nx, double2* __restrict__ dst) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nx) return;
  const float4 v = src[j];
  dst[j] = make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}

// co-resident CTAs per SM at `smem` bytes of dynamic shared memory
int march_dw_blocks_per_sm(size_t smem) {
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_march_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march_dw, kDwThreads, smem) != cudaSuccess) return 0;
  return per;
}

int march_dw_max_grid(int device) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march_dw, kDwThreads, 0);
  return sms * (per > 0 ? per : 0);
}

cudaError_t launch_tables_dw(const cd* etab, const cd* phitab, const cd* rowscal, const cd* detab, double C,
                             int64_t nt, int64_t nphi, int D, float4* etabC, float4* phitab_dw, float4* rowscal_dw,
                             float4* detab_dw, cudaStream_t s) {
  int64_t n = nphi > nt + D ? nphi : nt + D;
  k_tables_dw<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(etab, phitab, rowscal, detab, C, nt, nphi, D, etabC,
                                                           phitab_dw, rowscal_dw, detab_dw);
  return cudaGetLastError();
}

cudaError_t launch_march_dw(const DwArgs& a, int grid, size_t smem, cudaStream_t s) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_march_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  void* args[] = {const_cast<DwArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)k_march_dw, dim3(grid), dim3(kDwThreads), args, smem, s);
}

cudaError_t launch_norms_rows(const double* partials, int grid, int64_t n_begin, int64_t n_end, const cd* etab,
                             const cd* phitab, const cd* etab2, const cd* phitab2, double C, double delta,
                             double* norms, cudaStream_t s) {
  const int64_t rows = n_end - n_begin;
  if (rows <= 0) return cudaSuccess;
  k_norms_rows<<<(unsigned)((rows + 127) / 128), 128, 0, s>>>(partials, grid, n_begin, n_end, etab, phitab, etab2,
                                                              phitab2, C, delta, norms);
  return cudaGetLastError();
}

cudaError_t launch_row_dw(const float4* src, int64_t nx, double2* dst, cudaStream_t s) {
  k_row_dw<<<(unsigned)((nx + 255) / 256), 256, 0, s>>>(src, nx, dst);
  return cudaGetLastError();
}

}  // namespace fdtd
