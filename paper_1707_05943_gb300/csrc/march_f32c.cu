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
// (shared memory, the CTA edge in a two-slot global array) until the next row
// consumes it at column m+1.  The boundary tables, the exact boundary value
// psi(-a, t) at the first column and the norm reduction stay FP64.
//
// Work layout: thread-block clusters of up to 16 CTAs x 512 threads.  A
// cluster takes the next instance from a queue (largest first), splits its
// columns over its CTAs (weighting the costlier region -a < x <= 3a), and
// marches the instance's rows with one cluster barrier per row; rows n-1, n-D
// and n-D-1 are then complete.  Inside a CTA each thread owns a contiguous
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

// S without the a_lo and c2 y_{m-1} parts, and a_hi, for a column of -a < x <= 3a
__device__ __noinline__ float2 rhs_general32(const InstDesc& I, int64_t n, int nslot, int64_t j, float2 R2,
                                             float2* a_hi) {
  const int D = I.D, Dh = D >> 1;
  const int64_t m = j - Dh + 1;
  float2 a = psi_any32(I, n, nslot, n - 1, m - 1);
  *a_hi = a;
  float2 S = mulc(I.d1, a);
  S = fmac(I.c2, psi_any32(I, n, nslot, n - 1, m), S);
  if (n >= D + 1) {
    float2 sq = add(add(psi_any32(I, n, nslot, n - D, m - D), psi_any32(I, n, nslot, n - D, m - D - 1)),
                    add(psi_any32(I, n, nslot, n - D - 1, m - D), psi_any32(I, n, nslot, n - D - 1, m - D - 1)));
    S = fmac(I.c3, sq, S);
  }
  const int64_t r2 = n - m - Dh;
  if (r2 >= 0) {
    float w = (r2 == 0) ? 0.5f : 1.0f;
    float2 bl = add(psi_any32(I, n, nslot, r2, -m - D), psi_any32(I, n, nslot, r2, -m - D + 1));
    float2 br = add(psi_any32(I, n, nslot, r2, -m), psi_any32(I, n, nslot, r2, -m + 1));
    S = fmac(I.gs, scal(w, sub(bl, br)), S);
    S = fmac(R2, I.phitab32[r2], S);
  }
  if (m >= Dh + 1) {
    const int64_t r3 = n - m + Dh;
    if (r3 >= 0) {
      float w = (r3 == 0) ? 0.5f : 1.0f;
      float2 bl = add(psi_any32(I, n, nslot, r3, D - m), psi_any32(I, n, nslot, r3, D - m + 1));
      float2 br = add(psi_any32(I, n, nslot, r3, -m), psi_any32(I, n, nslot, r3, -m + 1));
      S = fmac(I.gs, scal(w, sub(bl, br)), S);
    }
  }
  return S;
}

__device__ __forceinline__ float2 rhs_bulk32(const InstDesc& I, const RowF& R, int64_t j, float2* a_hi) {
  const int D = I.D;
  float2 a = ldr(R.row1 + j - 1);
  *a_hi = a;
  float2 S = mulc(I.d1, a);
  S = fmac(I.c2, ldr(R.row1 + j), S);
  if (R.rowD) {
    float2 hn = add(ldr(R.rowD + j - D - 1), ldr(R.rowD + j - D));
    if (R.rowD1) {
      float2 hp = (R.hs && !R.cold) ? R.hs[j - R.hbase] : add(ldr(R.rowD1 + j - D - 1), ldr(R.rowD1 + j - D));
      S = fmac(I.c3, add(hn, hp), S);
    }
    if (R.hs) R.hs[j - R.hbase] = hn;
  }
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

// columns of CTA `rank` of `C` for an instance: split by cost
__device__ __forceinline__ void cta_range(const InstDesc& I, int rank, int C, int64_t* lo, int64_t* hi) {
  const int64_t G2 = (2 * (int64_t)I.D < I.nx) ? 2 * (int64_t)I.D : I.nx;
  const int64_t wm = I.mid_weight;
  const int64_t W = wm * G2 + (I.nx - G2);
  auto inv = [&](int64_t x) { return x <= wm * G2 ? (x + wm - 1) / wm : G2 + (x - wm * G2); };
  *lo = inv(W * rank / C);
  *hi = inv(W * (rank + 1) / C);
}

__global__ void __launch_bounds__(kF32Threads, 1)
    k_march_f32c(const InstDesc* __restrict__ insts, const int* __restrict__ order, int ninst,
                 unsigned int* queue, SyncWords* sync) {
  constexpr int P = kF32P;
  extern __shared__ float2 smem[];
  __shared__ float2 s_last[kF32Threads];
  __shared__ int s_len[kF32Threads];
  __shared__ float2 s_carry;
  __shared__ float2 s_halo[kMaxTrunc];
  __shared__ double s_red[kF32Threads / 32];
  __shared__ int s_inst;

  const int tid = threadIdx.x;
  const unsigned rank = cluster_rank(), C = cluster_size();

  for (;;) {
    // the cluster's next instance
    if (rank == 0 && tid == 0) {
      unsigned q = atomicAdd(queue, 1u);
      s_inst = (q < (unsigned)ninst) ? order[q] : -1;
    }
    cluster_sync_all();
    const int inst = ld_dsmem_i32(&s_inst, 0);
    cluster_sync_all();  // s_inst is read by every CTA before rank 0 may overwrite it
    if (inst < 0) break;
    const InstDesc& I = insts[inst];
    const int64_t n_begin = I.range[0], n_end = I.range[1];
    if (n_begin >= n_end) continue;
    const int D = I.D;

    int64_t j_lo, j_hi;
    cta_range(I, (int)rank, (int)C, &j_lo, &j_hi);
    const int64_t L = j_hi - j_lo;
    const int64_t G2 = (2 * (int64_t)D < I.nx) ? 2 * (int64_t)D : I.nx;
    int64_t s0, s1;
    if (j_lo >= G2) {
      const int64_t seg = ((L + kF32Threads - 1) / kF32Threads) | 1;
      s0 = j_lo + (int64_t)tid * seg;
      if (s0 > j_hi) s0 = j_hi;
      s1 = (s0 + seg < j_hi) ? s0 + seg : j_hi;
    } else {
      const int64_t wm = I.mid_weight;
      auto cumw = [&](int64_t j) { return j <= G2 ? wm * j : wm * G2 + (j - G2); };
      auto inv = [&](int64_t x) { return x <= wm * G2 ? (x + wm - 1) / wm : G2 + (x - wm * G2); };
      const int64_t W0 = cumw(j_lo), W1 = cumw(j_hi);
      s0 = inv(W0 + (W1 - W0) * tid / kF32Threads);
      s1 = inv(W0 + (W1 - W0) * (tid + 1) / kF32Threads);
    }
    const int64_t h0 = (j_lo - I.khalo > 0) ? j_lo - I.khalo : 0;
    const int nh = (int)(j_lo - h0);
    // shared memory: pair sums (khalo + L), then two slots of a_lo (L + 1 each)
    const int64_t hcap = I.smem_cols;
    float2* hs = smem;
    float2* es0 = smem + hcap;
    float2* es1 = es0 + (hcap + 1);
    const bool reuse = (L + nh <= hcap);
    s_len[tid] = (int)(s1 - s0);
    // a_lo of row n_begin-1, saved by the previous launch
    {
      float2* es = ((n_begin - 1) & 1) ? es1 : es0;
      for (int64_t j = j_lo + tid; j <= j_hi && reuse; j += kF32Threads)
        es[j - j_lo] = (j < I.nx && j - 1 >= 0) ? I.lo_g[j - 1] : f2(0.f, 0.f);
    }
    __syncthreads();

    for (int64_t n = n_begin; n < n_end; ++n) {
      RowF R;
      R.n = n;
      R.nslot = (int)(n % I.R);
      R.row1 = I.ring + (int64_t)((n - 1) % I.R) * I.stride;
      R.rowD = (n >= D) ? I.ring + (int64_t)((n - D) % I.R) * I.stride : nullptr;
      R.rowD1 = (n >= D + 1) ? I.ring + (int64_t)((n - D - 1) % I.R) * I.stride : nullptr;
      float2* row0 = I.ring + (int64_t)R.nslot * I.stride;
      float2* snap =
          (I.snaps && I.tstep >= 0 && n % (I.tstep + 1) == 0) ? I.snaps + (n / (I.tstep + 1)) * I.nx : nullptr;
      R.R1 = I.rowscal32[2 * n];
      R.R2 = I.rowscal32[2 * n + 1];
      R.hs = reuse ? hs : nullptr;
      R.hbase = h0;
      R.cold = (n == n_begin);
      float2* es_rd = ((n - 1) & 1) ? es1 : es0;  // a_lo of row n-1, by consumer column
      float2* es_wr = (n & 1) ? es1 : es0;        // a_lo for row n+1

      if (tid < 32 && j_lo < j_hi) {
        // the CTA's first column: the exact boundary value (first CTA) or the left CTA's edge
        if (tid == 0) {
          if (j_lo == 0) {
            const cd ex = I.C * (I.phitab[n - 1] * I.etab[n - 1]);  // psi(-a, (n-1) delta), FP64
            es_rd[0] = f2((float)(ex.re - (double)(float)ex.re), (float)(ex.im - (double)(float)ex.im));
          } else {
            es_rd[0] = I.lo_edge[((n - 1) & 1) * kClusterMax + rank - 1];
          }
        }
        for (int c = tid; c < nh; c += 32) {
          float2 ah;
          float2 S = rhs32(I, R, h0 + c, &ah);
          s_halo[c] = add(ah, S);
        }
        __syncwarp();
        if (tid == 0) {
          float2 y = f2(0.f, 0.f);
          if (h0 == 0) {
            const cd ex = I.C * (I.phitab[n] * I.etab[n]);  // psi(-a, n delta)
            y = f2((float)ex.re, (float)ex.im);
          }
          for (int c = 0; c < nh; ++c) y = fmac(I.c2, y, s_halo[c]);
          s_carry = y;
        }
      }
      __syncthreads();  // es_rd[0] and s_carry ready

      // pass A
      float2 ahv[P], Sv[P];
      float2 y = f2(0.f, 0.f);
      float nacc = 0.f;
#pragma unroll
      for (int v = 0; v < P; ++v) {
        const int64_t j = s0 + v;
        ahv[v] = f2(0.f, 0.f);
        Sv[v] = f2(0.f, 0.f);
        if (j < s1) {
          float2 ah;
          float2 S = rhs32(I, R, j, &ah);
          if (j == 0) ah = f2((float)(I.C * (I.phitab[n - 1] * I.etab[n - 1]).re),
                              (float)(I.C * (I.phitab[n - 1] * I.etab[n - 1]).im));
          S = add(S, es_rd[j - j_lo]);
          S = fmac(I.c2, y, S);
          ahv[v] = ah;
          Sv[v] = S;
          y = add(ah, S);
        }
      }
      for (int64_t j = s0 + P; j < s1; ++j) {
        float2 ah;
        float2 S = rhs32(I, R, j, &ah);
        S = add(S, es_rd[j - j_lo]);
        S = fmac(I.c2, y, S);
        if (j - s0 < I.kfix) {
          // still receives the carry: park S and a_hi in the slots this thread fills in pass B
          row0[j] = S;
          es_wr[j + 1 - j_lo] = ah;
          y = add(ah, S);
        } else {
          float2 s, e;
          two_sum(ah.x, S.x, s.x, e.x);
          two_sum(ah.y, S.y, s.y, e.y);
          row0[j] = s;
          if (snap) snap[j] = s;
          es_wr[j + 1 - j_lo] = e;
          nacc = fmaf(s.x, s.x, nacc);
          nacc = fmaf(s.y, s.y, nacc);
          y = s;
        }
      }
      s_last[tid] = (s0 < s1) ? y : f2(0.f, 0.f);
      __syncthreads();

      // pass B: carry, correction of the first kfix columns, TwoSum
      if (s0 < s1) {
        float2 carry = f2(0.f, 0.f), ap = f2(1.f, 0.f);
        for (int s = 1; s <= tid + 1; ++s) {
          if (tid - s >= 0) {
            carry = fmac(ap, s_last[tid - s], carry);
            const int lu = s_len[tid - s];
            ap = mulc(ap, (lu <= kF32MaxTrunc) ? I.c2pow[lu] : f2(0.f, 0.f));
            if (ap.x * ap.x + ap.y * ap.y < 2.2e-16f) break;  // (2^-26)^2
          } else {
            carry = fmac(ap, s_carry, carry);
          }
        }
#pragma unroll
        for (int v = 0; v < P; ++v) {
          const int64_t j = s0 + v;
          if (j < s1) {
            float2 S = (v < I.kfix) ? fmac(I.c2pow[v + 1], carry, Sv[v]) : Sv[v];
            float2 s, e;
            two_sum(ahv[v].x, S.x, s.x, e.x);
            two_sum(ahv[v].y, S.y, s.y, e.y);
            row0[j] = s;
            if (snap) snap[j] = s;
            es_wr[j + 1 - j_lo] = e;
            nacc = fmaf(s.x, s.x, nacc);
            nacc = fmaf(s.y, s.y, nacc);
          }
        }
        for (int v = P; v < I.kfix && s0 + v < s1; ++v) {
          const int64_t j = s0 + v;
          const float2 S = fmac(I.c2pow[v + 1], carry, row0[j]);
          const float2 ah = es_wr[j + 1 - j_lo];
          float2 s, e;
          two_sum(ah.x, S.x, s.x, e.x);
          two_sum(ah.y, S.y, s.y, e.y);
          row0[j] = s;
          if (snap) snap[j] = s;
          es_wr[j + 1 - j_lo] = e;
          nacc = fmaf(s.x, s.x, nacc);
          nacc = fmaf(s.y, s.y, nacc);
        }
        if (s1 == j_hi) {  // the CTA's last column: its a_lo goes to the next CTA
          I.lo_edge[(n & 1) * kClusterMax + rank] = es_wr[j_hi - j_lo];
        }
      }

      // norm partial: FP32 within a thread (its few columns), FP64 from there on
      double dn = (double)nacc;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dn += __shfl_down_sync(0xffffffffu, dn, o);
      if ((tid & 31) == 0) s_red[tid >> 5] = dn;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kF32Threads / 32; ++w) t += s_red[w];
        if (j_hi == I.nx && j_lo < j_hi) {
          float2 l = row0[I.nx - 1];
          t -= 0.5 * ((double)l.x * l.x + (double)l.y * l.y);
        }
        I.partials[(n & 1) * kClusterMax + rank] = t;
      }
      cluster_sync_all();
      if (rank == 0 && tid == 0) {
        const cd ex = I.C * (I.phitab[n] * I.etab[n]);
        double t = 0.5 * cabs2(ex);
        for (unsigned b = 0; b < C; ++b) t += I.partials[(n & 1) * kClusterMax + b];
        I.norms[n] = I.delta * t;
      }
    }
    // save a_lo of the last row for the next launch
    {
      float2* es = ((n_end - 1) & 1) ? es1 : es0;
      for (int64_t j = j_lo + 1 + tid; j <= j_hi; j += kF32Threads)
        if (j - 1 < I.nx) I.lo_g[j - 1] = es[j - j_lo];
    }
    cluster_sync_all();  // lo_g and lo_edge complete before any CTA moves on
  }
  (void)sync;
}

// FP32 copies of the boundary tables an instance's march reads
__global__ void k_tables32(InstDesc I, const cd* detab, const cd* rowscal) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  auto cv = [](cd v) { return make_float2((float)v.re, (float)v.im); };
  if (i < I.nt) {
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

size_t march_f32c_smem(int64_t cols) { return sizeof(float2) * (size_t)(3 * cols + 2); }

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

cudaError_t launch_march_f32c(const InstDesc* insts, const int* order, int ninst, unsigned int* queue,
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
  return cudaLaunchKernelEx(&cfg, k_march_f32c, insts, order, ninst, queue, sync);
}

}  // namespace fdtd
