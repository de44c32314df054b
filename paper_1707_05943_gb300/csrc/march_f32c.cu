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
// produced it, recovered exactly by TwoSum(a_hi, S) (Knuth) and kept on chip
// (a two-slot array by row parity, L2-resident) until the next row consumes it
// at column m+1.  The boundary tables, the exact boundary value
// psi(-a, t) at the first column and the norm reduction stay FP64.
//
// Work layout: thread-block clusters of up to 8 CTAs x 256 threads.  A
// cluster takes the next work item from a queue (largest first): either one
// wide instance, whose columns it splits over its CTAs (the costlier region
// -a < x <= 3a on CTAs of its own when it is worth one, see cta_range) and
// whose rows it marches with one cluster barrier per row, or up to one narrow
// instance per CTA, marched with CTA barriers only.
// Either way rows n-1, n-D and n-D-1 are complete when row n starts.  Inside a CTA each thread owns a contiguous
// segment and runs the recurrence y_m = c2 y_{m-1} + r_m over it from a zero
// carry; after a CTA barrier it takes its carry from the threads before it
// and corrects its first kfix columns (|c2|^kfix < 2^-26, below FP32
// rounding).  Clusters never wait on each other: the queue counter is the only
// state they share, so the launch needs no co-residency.
#include <cuda_runtime.h>

#include "fdtd_internal.cuh"

namespace fdtd {

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

// TwoSum: s = fl(a+b), e = (a+b) - s exactly (round to nearest, no FMA involved)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float2 ldr(const float2* p) { return *p; }

__device__ __forceinline__ float2 psi_left32(const InstDesc& I, int64_t r, int64_t c) {
  const int Dh = I.D >> 1;
  return scal((float)I.C, mulc(I.phitab32[r - c - Dh], I.etab32[r]));
}

__device__ __forceinline__ float2 psi_any32(const InstDesc& I, int64_t n, int nslot, int64_t r, int64_t c) {
  const int Dh = I.D >> 1;
  if (c <= -Dh) return psi_left32(I, r, c);
  int slot = nslot - (int)(n - r);
  if (slot < 0) slot += I.R;
  return ldr(&I.ring[(int64_t)slot * I.stride + (c + Dh - 1)]);
}

struct RowF {
  int64_t n;
  int nslot;
  const float2* row1;
  const float2* rowD;
  const float2* rowD1;
  float2 R1, R2;
  float2* hs;
  int64_t hbase;
  bool cold;
};

// S without the a_lo and c2 y_{m-1} parts, and a_hi, for a column of -a < x <= 3a.
// Its up to 14 reads (stencil, delay square, the mirror bars of lines 2-3) go
// to scattered rows; they are all issued before any is used.
__device__ __noinline__ float2 rhs_general32(const InstDesc& I, int64_t n, int nslot, int64_t j, float2 R2,
                                             float2* a_hi) {
  const int D = I.D, Dh = D >> 1;
  const int64_t m = j - Dh + 1;
  const int64_t r2 = n - m - Dh, r3 = n - m + Dh;
  const bool dl = (n >= D + 1), s2 = (r2 >= 0), s3 = (m >= Dh + 1) && (r3 >= 0);
  int64_t rr[14], cc[14];
  bool ok[14];
  rr[0] = n - 1; cc[0] = m - 1; ok[0] = true;
  rr[1] = n - 1; cc[1] = m; ok[1] = true;
  rr[2] = n - D; cc[2] = m - D; rr[3] = n - D; cc[3] = m - D - 1;
  rr[4] = n - D - 1; cc[4] = m - D; rr[5] = n - D - 1; cc[5] = m - D - 1;
  ok[2] = ok[3] = ok[4] = ok[5] = dl;
  rr[6] = r2; cc[6] = -m - D; rr[7] = r2; cc[7] = -m - D + 1; rr[8] = r2; cc[8] = -m; rr[9] = r2; cc[9] = -m + 1;
  ok[6] = ok[7] = ok[8] = ok[9] = s2;
  rr[10] = r3; cc[10] = D - m; rr[11] = r3; cc[11] = D - m + 1; rr[12] = r3; cc[12] = -m; rr[13] = r3; cc[13] = -m + 1;
  ok[10] = ok[11] = ok[12] = ok[13] = s3;
  // unconditional loads (indices clamped into the tables and the ring), selected below
  float2 ph[14], ev[14], rg[14];
#pragma unroll
  for (int k = 0; k < 14; ++k) {
    int64_t ai = rr[k] - cc[k] - Dh;
    ai = ai < 0 ? 0 : (ai >= I.nphi ? I.nphi - 1 : ai);
    int64_t ei = rr[k] < 0 ? 0 : (rr[k] >= I.nt ? I.nt - 1 : rr[k]);
    int lag = (int)(n - rr[k]);
    lag = lag < 0 ? 0 : (lag >= I.R ? I.R - 1 : lag);
    int slot = nslot - lag;
    if (slot < 0) slot += I.R;
    int64_t ci = cc[k] + Dh - 1;
    ci = ci < 0 ? 0 : (ci >= I.nx ? I.nx - 1 : ci);
    ph[k] = I.phitab32[ai];
    ev[k] = I.etab32[ei];
    rg[k] = ldr(&I.ring[(int64_t)slot * I.stride + ci]);
  }
  const float2 chi = I.phitab32[s2 ? r2 : 0];
  float2 v[14];
#pragma unroll
  for (int k = 0; k < 14; ++k)
    v[k] = !ok[k] ? f2(0.f, 0.f) : ((cc[k] <= -Dh) ? scal((float)I.C, mulc(ph[k], ev[k])) : rg[k]);
  *a_hi = v[0];
  float2 S = mulc(I.d1, v[0]);
  S = fmac(I.c2, v[1], S);
  float2 L = mulc(I.d1lo, v[0]);  // the coefficients' low parts
  L = fmac(I.c2lo, v[1], L);
  if (dl) {
    const float2 sq = add(add(v[2], v[3]), add(v[4], v[5]));
    S = fmac(I.c3, sq, S);
    L = fmac(I.c3lo, sq, L);
  }
  S = add(S, L);
  if (s2) {
    const float w = (r2 == 0) ? 0.5f : 1.0f;
    S = fmac(I.gs, scal(w, sub(add(v[6], v[7]), add(v[8], v[9]))), S);
    S = fmac(R2, chi, S);
  }
  if (s3) {
    const float w = (r3 == 0) ? 0.5f : 1.0f;
    S = fmac(I.gs, scal(w, sub(add(v[10], v[11]), add(v[12], v[13]))), S);
  }
  return S;
}

__device__ __forceinline__ float2 rhs_bulk32(const InstDesc& I, const RowF& R, int64_t j, float2* a_hi) {
  const int D = I.D;
  float2 a = ldr(R.row1 + j - 1);
  *a_hi = a;
  const float2 b = ldr(R.row1 + j);
  float2 S = mulc(I.d1, a);
  S = fmac(I.c2, b, S);
  float2 L = fmac(I.c2lo, b, mulc(I.d1lo, a));
  if (R.rowD) {
    float2 hn = add(ldr(R.rowD + j - D - 1), ldr(R.rowD + j - D));
    if (R.rowD1) {
      float2 hp = (R.hs && !R.cold) ? R.hs[j - R.hbase] : add(ldr(R.rowD1 + j - D - 1), ldr(R.rowD1 + j - D));
      const float2 sq = add(hn, hp);
      S = fmac(I.c3, sq, S);
      L = fmac(I.c3lo, sq, L);
    }
    if (R.hs) R.hs[j - R.hbase] = hn;
  }
  S = add(S, L);
  const int64_t i = R.n - j - 1 + D;  // r2 + D
  if (i >= 0) {
    S = fmac(R.R1, I.detab32[i], S);
    if (i >= D) S = fmac(R.R2, I.phitab32[i - D], S);
  }
  return S;
}

__device__ __forceinline__ float2 rhs32(const InstDesc& I, const RowF& R, int64_t j, float2* a_hi) {
  if (j >= 2 * (int64_t)I.D) return rhs_bulk32(I, R, j, a_hi);
  return rhs_general32(I, R.n, R.nslot, j, R.R2, a_hi);
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(r));
  return r;
}
// read a 32-bit word from CTA `rank`'s shared memory (same offset)
__device__ __forceinline__ int ld_dsmem_i32(const int* local, unsigned rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(local), ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(ra) : "r"(a), "r"(rank));
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];\n" : "=r"(v) : "r"(ra) : "memory");
  return v;
}

__device__ __forceinline__ float ld_dsmem_f32(const float* local, unsigned rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(local), ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(ra) : "r"(a), "r"(rank));
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];\n" : "=f"(v) : "r"(ra) : "memory");
  return v;
}

// columns of CTA `rank` of `C` for an instance.  The first G2 = 2D columns
// (-a < x <= 3a) cost mid_weight bulk columns each.  When they are worth about
// one CTA or more, whole CTAs take them (split evenly) and the others the bulk
// (split evenly), so that no CTA mixes the two kinds; otherwise one cost-weighted
// split.  The host mirrors this rule to size shared memory.
__device__ __forceinline__ void cta_range(const InstDesc& I, int rank, int C, int64_t* lo, int64_t* hi) {
  const int64_t G2 = (2 * (int64_t)I.D < I.nx) ? 2 * (int64_t)I.D : I.nx;
  const int64_t wm = I.mid_weight;
  const int64_t W = wm * G2 + (I.nx - G2);
  int64_t g = (2 * (int64_t)C * wm * G2 + W) / (2 * W);
  if (g > C - 1) g = C - 1;
  if (g >= 1 && I.nx > G2) {
    if (rank < g) {
      *lo = G2 * rank / g;
      *hi = G2 * (rank + 1) / g;
    } else {
      const int64_t r = rank - g, Cb = C - g;
      *lo = G2 + (I.nx - G2) * r / Cb;
      *hi = G2 + (I.nx - G2) * (r + 1) / Cb;
    }
    return;
  }
  auto inv = [&](int64_t x) { return x <= wm * G2 ? (x + wm - 1) / wm : G2 + (x - wm * G2); };
  *lo = inv(W * rank / C);
  *hi = inv(W * (rank + 1) / C);
}

// ---- TMA bulk copies into shared memory (1D), completion on an mbarrier ----
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned a = (unsigned)__cvta_generic_to_shared(bar), ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// copy `bytes` (multiple of 16) from 16-byte aligned global memory to shared memory
__device__ __forceinline__ void tma_load_1d(void* sdst, const void* gsrc, unsigned bytes, uint64_t* bar) {
  unsigned d = (unsigned)__cvta_generic_to_shared(sdst), m = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(d),
               "l"(gsrc), "r"(bytes), "r"(m)
               : "memory");
}

// A staged slice: global elements [g0, g1) of a float2 array start at smem
// element `off` (0 or 1: the copy starts on an even element, 16-byte aligned).
struct Slice {
  float2* s;
  int off;
  int64_t g0;
  __device__ __forceinline__ float2 at(int64_t g) const { return s[g - g0 + off]; }
};

// plan the copy of global elements [g0, g1) into `dst`: the copy starts on an
// even element (16-byte aligned) and moves an even number of elements
struct Copy {
  float2* dst;
  const float2* src;
  unsigned bytes;
};
__device__ __forceinline__ Copy plan_copy(Slice& sl, float2* dst, const float2* src, int64_t g0, int64_t g1) {
  const int64_t a = g0 & ~int64_t(1), b = (g1 + 1) & ~int64_t(1);
  sl.s = dst;
  sl.off = (int)(g0 - a);
  sl.g0 = g0;
  return Copy{dst, src + a, (unsigned)((b - a) * sizeof(float2))};
}

constexpr int kBlk = 2048;        // bulk columns staged per block
constexpr int kStageCols = kBlk + 4;

__global__ void __launch_bounds__(kF32Threads, 1)
    k_march_f32c(const InstDesc* __restrict__ insts, const WorkItem* __restrict__ items, int nitems,
                 unsigned int* queue, SyncWords* sync) {
  extern __shared__ __align__(128) float2 smem[];
  __shared__ float2 s_last[kF32Threads];
  __shared__ int s_len[kF32Threads];
  __shared__ float2 s_carry[2];  // carry into a block, by block parity: a block's pass B reads one slot
                                 // while the thread ending that block writes the other
  __shared__ float2 s_halo[kMaxTrunc];
  __shared__ float s_red[2][kF32Threads / 32];
  __shared__ int s_inst;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ __align__(16) InstDesc s_I;  // the instance's descriptor: no global store can alias it

  const int tid = threadIdx.x;
  const unsigned rank = cluster_rank(), C = cluster_size();
  // shared memory: 6 staging slices, then the pair sums of the CTA's columns
  float2* st_a1 = smem;
  float2* st_ad = st_a1 + kStageCols;
  float2* st_ad1 = st_ad + kStageCols;
  float2* st_lo = st_ad1 + kStageCols;
  float2* st_de = st_lo + kStageCols;
  float2* st_ph = st_de + kStageCols;
  float2* o_hi = st_ph + kStageCols;  // block results: hi (or parked S), remainder (or parked a_hi)
  float2* o_e = o_hi + kStageCols;
  float2* hs_base = o_e + kStageCols;
  if (tid == 0) mbar_init(&s_bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  __syncthreads();
  unsigned bar_phase = 0;

  for (;;) {
    // the cluster's next work item: one wide instance for the whole cluster, or
    // up to C narrow instances, one per CTA ("solo": CTA barriers only)
    if (rank == 0 && tid == 0) {
      unsigned q = atomicAdd(queue, 1u);
      s_inst = (q < (unsigned)nitems) ? (int)q : -1;
    }
    cluster_sync_all();
    const int item = ld_dsmem_i32(&s_inst, 0);
    cluster_sync_all();  // s_inst is read by every CTA before rank 0 may overwrite it
    if (item < 0) break;
    const WorkItem& Wk = items[item];
    const bool solo = Wk.solo != 0;
    const int inst = solo ? ((rank < (unsigned)Wk.count) ? Wk.inst[rank] : -1) : Wk.inst[0];
    const unsigned rank_e = solo ? 0u : rank, C_e = solo ? 1u : C;
    if (inst >= 0) {
      const int* src = reinterpret_cast<const int*>(&insts[inst]);
      int* dst = reinterpret_cast<int*>(&s_I);
      for (int k = tid; k < (int)(sizeof(InstDesc) / sizeof(int)); k += kF32Threads) dst[k] = src[k];
    }
    __syncthreads();
    if (inst >= 0 && s_I.range[0] < s_I.range[1]) {
      const InstDesc& I = s_I;
      const int64_t n_begin = I.range[0], n_end = I.range[1];
      const int D = I.D;
      int64_t j_lo, j_hi;
      cta_range(I, (int)rank_e, (int)C_e, &j_lo, &j_hi);
      const int64_t G2 = (2 * (int64_t)D < I.nx) ? 2 * (int64_t)D : I.nx;
      const int64_t h0 = (j_lo - I.khalo > 0) ? j_lo - I.khalo : 0;
      const int nh = (int)(j_lo - h0);
      const bool reuse = (j_hi - j_lo + nh <= I.smem_cols);  // pair sums kept in shared memory
      float2* hs = reuse ? hs_base : nullptr;

      int slot = (int)(n_begin % I.R);
      int64_t snap_ctr = (I.tstep >= 0) ? n_begin % (I.tstep + 1) : -1;
      for (int64_t n = n_begin; n < n_end; ++n) {
        auto back = [&](int k) { int t = slot - k; return t < 0 ? t + I.R : t; };
        RowF R;
        R.n = n;
        R.nslot = slot;
        R.row1 = I.ring + (int64_t)back(1) * I.stride;
        R.rowD = (n >= D) ? I.ring + (int64_t)back(D) * I.stride : nullptr;
        R.rowD1 = (n >= D + 1) ? I.ring + (int64_t)back(D + 1) * I.stride : nullptr;
        float2* row0 = I.ring + (int64_t)slot * I.stride;
        float2* snap = (snap_ctr == 0) ? I.snaps + (n / (I.tstep + 1)) * I.nx : nullptr;
        R.R1 = I.rowscal32[2 * n];
        R.R2 = I.rowscal32[2 * n + 1];
        R.hs = hs;
        R.hbase = h0;
        R.cold = (n == n_begin);
        float2* es_rd = I.lo + (int64_t)((n - 1) & 1) * I.lo_pitch;
        float2* es_wr = I.lo + (int64_t)(n & 1) * I.lo_pitch;
        float nacc = 0.f;

        // carry into the CTA's first column: psi(-a) for the first CTA, else the
        // recurrence over khalo columns to its left (warp 0)
        if (tid < 32 && j_lo < j_hi) {
          if (tid == 0 && j_lo == 0) es_rd[0] = I.bnd32[2 * (n - 1) + 1];  // thread 0 owns column 0
          for (int c = tid; c < nh; c += 32) {
            float2 ah;
            float2 S = rhs32(I, R, h0 + c, &ah);
            s_halo[c] = add(ah, S);
          }
          __syncwarp();
          if (tid == 0) {
            float2 yh = (h0 == 0) ? I.bnd32[2 * n] : f2(0.f, 0.f);
            for (int c = 0; c < nh; ++c) yh = fmac(I.c2lo, yh, fmac(I.c2, yh, s_halo[c]));
            s_carry[0] = yh;
          }
        }

        // blocks: first the columns of -a < x <= 3a (read in place, cost-weighted
        // over the threads), then x > 3a in staged blocks of kBlk
        // the six staged slices of a bulk block [b0, b1): rows n-1, n-D, n-D-1, the
        // remainders of row n-1, and the source tables; thread 0 arms the barrier
        // with their bytes and issues the copies
        auto stage = [&](int64_t b0, int64_t b1, Slice& A1, Slice& AD, Slice& AD1, Slice& LO, Slice& DE,
                         Slice& PH) {
          const int64_t ib = n - b1 + D;  // detab index of the block's last column
          const int64_t ilo = (ib > 0) ? ib : 0, ihi = n - b0 + D;        // detab [ilo, ihi)
          const int64_t plo = (ib - D > 0) ? ib - D : 0, phi_ = n - b0;  // phitab [plo, phi_)
          Copy cp[6];
          cp[0] = plan_copy(A1, st_a1, R.row1, b0 - 1, b1);
          cp[1] = R.rowD ? plan_copy(AD, st_ad, R.rowD, b0 - D - 1, b1 - D) : Copy{nullptr, nullptr, 0u};
          cp[2] = (R.rowD1 && (!hs || R.cold)) ? plan_copy(AD1, st_ad1, R.rowD1, b0 - D - 1, b1 - D)
                                               : Copy{nullptr, nullptr, 0u};
          cp[3] = plan_copy(LO, st_lo, es_rd, b0, b1);
          cp[4] = (ihi > ilo) ? plan_copy(DE, st_de, I.detab32, ilo, ihi) : Copy{nullptr, nullptr, 0u};
          cp[5] = (phi_ > plo) ? plan_copy(PH, st_ph, I.phitab32, plo, phi_) : Copy{nullptr, nullptr, 0u};
          if (tid == 0) {
            unsigned bytes = 0;
            for (int k = 0; k < 6; ++k) bytes += cp[k].bytes;
            asm volatile("fence.proxy.async;\n" ::: "memory");
            mbar_expect_tx(&s_bar, bytes);
            for (int k = 0; k < 6; ++k)
              if (cp[k].bytes) tma_load_1d(cp[k].dst, cp[k].src, cp[k].bytes, &s_bar);
          }
        };
        // a bulk block's copies may be issued while the block before it finishes
        // (pass B and the stores read only the output buffers)
        bool pre = false;
        Slice pA1, pAD, pAD1, pLO, pDE, pPH;
        int blk = 0;  // block index within the row (selects the carry slot)
        int64_t c0 = j_lo;
        while (c0 < j_hi) {
          const bool gen = (c0 < G2);
          const int64_t c1 = gen ? ((j_hi < G2) ? j_hi : G2) : ((c0 + kBlk < j_hi) ? c0 + kBlk : j_hi);
          const int64_t len = c1 - c0;
          // this thread's segment of the block
          int64_t t0, t1;
          if (!gen) {
            const int64_t seg = ((len + kF32Threads - 1) / kF32Threads) | 1;
            t0 = c0 + (int64_t)tid * seg;
            if (t0 > c1) t0 = c1;
            t1 = (t0 + seg < c1) ? t0 + seg : c1;
          } else if (len < kF32Threads) {
            // fewer columns than threads: one column each on the first `len` threads, so
            // that every carry in pass B crosses only non-empty segments
            t0 = (tid < len) ? c0 + tid : c1;
            t1 = (tid < len) ? t0 + 1 : c1;
          } else {
            t0 = c0 + len * tid / kF32Threads;
            t1 = c0 + len * (tid + 1) / kF32Threads;
          }
          s_len[tid] = (int)(t1 - t0);

          Slice A1, AD, AD1, LO, DE, PH;
          if (!gen) {
            if (pre) {
              A1 = pA1;
              AD = pAD;
              AD1 = pAD1;
              LO = pLO;
              DE = pDE;
              PH = pPH;
              pre = false;
            } else {
              stage(c0, c1, A1, AD, AD1, LO, DE, PH);
            }
            // bounded wait for the copies
            long long tw = clock64();
            while (!mbar_try_wait(&s_bar, bar_phase)) {
              if (clock64() - tw > 4000000000LL) {
                if (atomicCAS(&sync->status, 0u, (unsigned)FDTD_ERR_TIMEOUT) == 0u) sync->where = n;
                break;
              }
            }
            bar_phase ^= 1u;
          }

          // pass A: the segment from a zero carry; its first kfix columns are
          // parked (S, a_hi) until pass B adds the carry.  Results of a staged
          // block go to shared memory (o_hi: hi or parked S, o_e: remainder or
          // parked a_hi) and leave in coalesced stores after pass B; a block of
          // -a < x <= 3a writes its few columns in place.
          float2 y = f2(0.f, 0.f);
          int v = 0;
          float2* oh = gen ? row0 + c0 : o_hi;      // column j at oh[j - c0]
          float2* oe = gen ? es_wr + c0 + 1 : o_e;  // remainder of column j at oe[j - c0]
          auto emit = [&](int64_t j, float2 ah, float2 S) {
            if (v < I.kfix) {
              oh[j - c0] = S;
              oe[j - c0] = ah;
              y = add(ah, S);
            } else {
              float2 sv, e;
              two_sum(ah.x, S.x, sv.x, e.x);
              two_sum(ah.y, S.y, sv.y, e.y);
              oh[j - c0] = sv;
              oe[j - c0] = e;
              const float wt = (j == I.nx - 1) ? 0.5f : 1.0f;
              nacc = fmaf(wt * sv.x, sv.x, nacc);
              nacc = fmaf(wt * sv.y, sv.y, nacc);
              y = sv;
            }
            ++v;
          };
          if (gen) {
            for (int64_t j = t0; j < t1; ++j) {
              float2 ah;
              float2 S = rhs_general32(I, n, R.nslot, j, R.R2, &ah);
              if (j == 0) ah = I.bnd32[2 * (n - 1)];
              S = add(S, __ldcg(es_rd + j));
              emit(j, ah, fmac(I.c2lo, y, fmac(I.c2, y, S)));
            }
          } else {
            // block-relative 32-bit offsets: column j = c0 + k
            const bool d1 = (R.rowD1 != nullptr), dd = (R.rowD != nullptr);
            const bool use_hs = hs && !R.cold;
            const float2* a1s = A1.s + A1.off;                 // a_hi(k) = a1s[k], b(k) = a1s[k+1]
            const float2* ads = AD.s + AD.off;                 // row n-D: ads[k], ads[k+1]
            const float2* ad1s = AD1.s + AD1.off;
            const float2* los = LO.s + LO.off;
            const int kde = (int)(n - c0 - 1 + D);             // i(k) = kde - k
            const float2* des = DE.s + DE.off - DE.g0;         // detab32[i] = des[i]
            const float2* phs = PH.s + PH.off - PH.g0;         // phitab32[i - D] = phs[i - D]
            float2* hsb = hs ? hs + (c0 - h0) : nullptr;
            const int k0 = (int)(t0 - c0), k1 = (int)(t1 - c0);
            const int klast = (int)(I.nx - 1 - c0);
            const float2 d1c = I.d1, c2c = I.c2, c3c = I.c3, R1 = R.R1, R2 = R.R2;
            const float2 d1l = I.d1lo, c2l = I.c2lo, c3l = I.c3lo;
            const int kfix = I.kfix;
            for (int k = k0; k < k1; ++k) {
              const float2 a = a1s[k], b = a1s[k + 1];
              float2 S = mulc(d1c, a);
              S = fmac(c2c, b, S);
              float2 L = fmac(c2l, b, mulc(d1l, a));
              if (dd) {
                const float2 hn = add(ads[k], ads[k + 1]);
                if (d1) {
                  const float2 sq = add(hn, use_hs ? hsb[k] : add(ad1s[k], ad1s[k + 1]));
                  S = fmac(c3c, sq, S);
                  L = fmac(c3l, sq, L);
                }
                if (hsb) hsb[k] = hn;
              }
              S = add(S, L);
              const int i = kde - k;
              if (i >= 0) S = fmac(R1, des[i], S);
              if (i >= D) S = fmac(R2, phs[i - D], S);
              S = add(S, los[k]);
              S = fmac(c2l, y, fmac(c2c, y, S));
              if (v < kfix) {
                o_hi[k] = S;
                o_e[k] = a;
                y = add(a, S);
              } else {
                float2 sv, e;
                two_sum(a.x, S.x, sv.x, e.x);
                two_sum(a.y, S.y, sv.y, e.y);
                o_hi[k] = sv;
                o_e[k] = e;
                const float wt = (k == klast) ? 0.5f : 1.0f;
                nacc = fmaf(wt * sv.x, sv.x, nacc);
                nacc = fmaf(wt * sv.y, sv.y, nacc);
                y = sv;
              }
              ++v;
            }
          }
          s_last[tid] = (t0 < t1) ? y : f2(0.f, 0.f);
          __syncthreads();
          // the staging slices are free: issue the next bulk block's copies now
          if (!gen && c1 < j_hi) {
            stage(c1, (c1 + kBlk < j_hi) ? c1 + kBlk : j_hi, pA1, pAD, pAD1, pLO, pDE, pPH);
            pre = true;
          }

          // pass B: carry from the threads before (the block's carry-in for thread 0)
          if (t0 < t1) {
            float2 carry = f2(0.f, 0.f), ap = f2(1.f, 0.f);
            for (int s = 1; s <= tid + 1; ++s) {
              if (tid - s >= 0) {
                carry = fmac(ap, s_last[tid - s], carry);
                const int lu = s_len[tid - s];
                ap = mulc(ap, (lu <= kF32MaxTrunc) ? I.c2pow[lu] : f2(0.f, 0.f));
                if (ap.x * ap.x + ap.y * ap.y < 2.2e-16f) break;  // (2^-26)^2
              } else {
                carry = fmac(ap, s_carry[blk & 1], carry);
              }
            }
            const int nf = (I.kfix < (int)(t1 - t0)) ? I.kfix : (int)(t1 - t0);
            const int kb = (int)(t0 - c0), klast = (int)(I.nx - 1 - c0), kend = (int)(t1 - 1 - c0);
            float2 ylast = y;
#pragma unroll 4
            for (int u = 0; u < nf; ++u) {  // only the kfix parked columns take the carry
              const int k = kb + u;
              const float2 S = fmac(I.c2powlo[u + 1], carry, fmac(I.c2pow[u + 1], carry, oh[k]));
              const float2 A = oe[k];
              float2 sv, e;
              two_sum(A.x, S.x, sv.x, e.x);
              two_sum(A.y, S.y, sv.y, e.y);
              oh[k] = sv;
              oe[k] = e;
              const float wt = (k == klast) ? 0.5f : 1.0f;
              nacc = fmaf(wt * sv.x, sv.x, nacc);
              nacc = fmaf(wt * sv.y, sv.y, nacc);
              if (k == kend) ylast = sv;
            }
            if (t1 == c1) s_carry[(blk + 1) & 1] = ylast;  // carry into the next block
            if (gen && snap)
              for (int64_t jj = t0; jj < t1; ++jj) snap[jj] = row0[jj];
          }
          __syncthreads();  // block results complete
          if (!gen) {  // coalesced stores of the block
            float2* r0 = row0 + c0;
            float2* ew = es_wr + c0 + 1;
            float2* sp = snap ? snap + c0 : nullptr;
            for (int k = tid; k < (int)len; k += kF32Threads) {
              const float2 h = o_hi[k];
              r0[k] = h;
              ew[k] = o_e[k];
              if (sp) sp[k] = h;
            }
            __syncthreads();  // staging and output buffers free for the next block
          }
          c0 = c1;
          ++blk;
        }

        // norm: FP32 within a warp, FP64 across warps and CTAs
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nacc += __shfl_down_sync(0xffffffffu, nacc, o);
        if ((tid & 31) == 0) s_red[n & 1][tid >> 5] = nacc;
        if (solo) __syncthreads();
        else cluster_sync_all();
        if (rank_e == 0 && tid < 32) {
          // warp 0 of rank 0 gathers every warp's partial (local or over DSMEM) at once
          constexpr int nw = kF32Threads / 32;
          const int tot = (int)C_e * nw;
          double t = 0.0;
          for (int q = tid; q < tot; q += 32) {
            const float* pw = &s_red[n & 1][q % nw];
            t += (double)(solo ? *pw : ld_dsmem_f32(pw, (unsigned)(q / nw)));
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
          if (tid == 0) I.norms[n] = I.delta * (t + I.bnorm[n]);
        }
        slot = (slot + 1 == I.R) ? 0 : slot + 1;
        if (snap_ctr >= 0) snap_ctr = (snap_ctr == I.tstep) ? 0 : snap_ctr + 1;
      }
    }
    cluster_sync_all();  // the item is complete before any CTA of the cluster moves on
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

size_t march_f32c_smem(int64_t cols) { return sizeof(float2) * (size_t)(8 * kStageCols + cols); }

int march_f32c_max_clusters(int csize, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_march_f32c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return -1;
  if (csize > 8) cudaFuncSetAttribute(k_march_f32c, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(kF32Threads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  e = cudaOccupancyMaxActiveClusters(&n, (const void*)k_march_f32c, &cfg);
  return e == cudaSuccess ? n : -1;
}

cudaError_t launch_march_f32c(const InstDesc* insts, const WorkItem* items, int nitems, unsigned int* queue,
                              SyncWords* sync, int nclusters, int csize, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nclusters * csize);
  cfg.blockDim = dim3(kF32Threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_march_f32c, insts, items, nitems, queue, sync);
}

}  // namespace fdtd
