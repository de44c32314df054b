// march_f64.cu -- persistent FP64 march of Eq. 1 in x > -a.
//
// Update of the point (n, m) (top-right corner of the square centred at
// x_c = (m-1/2) delta, t_c = (n-1/2) delta; Eq. 3a-c for line 1 with the delay
// term written as in App. A, Eq. 4 bars for lines 2-3, line 4 at the centre):
//
//   psi[n][m] = c1 psi[n-1][m-1] + c2 (psi[n-1][m] + psi[n][m-1])
//             + c3 [n >= D+1] (psi[n-D][m-D] + psi[n-D][m-D-1] + psi[n-D-1][m-D] + psi[n-D-1][m-D-1])
//             + (1/A) (S2 + S3 + Schi),
//   c1 = (1/delta - W/4)/A, c2 = -(W/4)/A, c3 = (Gamma/8)/A, A = 1/delta + W/4.
//
// Everything except c2 psi[n][m-1] depends on earlier rows only, so a row is
// r_m (parallel over m) followed by the first-order recurrence
// y_m = c2 y_{m-1} + r_m.  |c2| = |W delta| / |4 + W delta| < 1, so a carry's
// influence dies as |c2|^k; the recurrence is carried exactly while that
// influence exceeds 2^-60 (kfix columns) and truncated beyond, which is below
// FP64 rounding.
//
// Work layout: one persistent cooperative CTA per SM.  CTA b owns the columns
// [colsplit[b], colsplit[b+1]) of every row; each of its threads owns one
// contiguous segment of them.  Per row a thread runs the recurrence over its
// segment from a zero carry, keeping the first kMarchP columns in registers
// and storing the rest (exact once kfix columns have passed).  After a CTA
// barrier the thread takes its carry from the local last values of the
// threads before it, adds c2^(v+1) carry to its first kfix columns, and
// stores them.  The carry into a CTA's first column is the recurrence run over
// khalo columns to its left (the exact boundary value psi(-a, t) for the first
// CTA).  Rows are not separated by a grid barrier: before row n a CTA waits
// (bounded) only until the CTAs it reads have completed the rows it reads from
// them, and until the CTAs that read it no longer need the ring slot of row n
// (RowDeps in fdtd_internal.cuh); the ring holds D + 2 + kRowSlack rows.  The
// per-row norm is summed from the CTAs' partials by a separate kernel after the
// launch, in a fixed order.
//
// The delay term needs psi[n-D][m-D-1] + psi[n-D][m-D] and the same pair on
// row n-D-1; the latter is the former of the previous row, so each column's
// pair sum is kept in shared memory from one row to the next.
//
// Reads of x <= -a use psi(x,t) = C phi(x-t) e(t) from the boundary tables.
// Beyond x > 3a every mirror read of lines 2-3 lands in x <= -a, and the
// sources collapse to R1(n) [E(r2) - E(r2+D)] + R2(n) phi(r2), r2 = n - m - D/2,
// E(r) = theta(r) e(r delta), with the bracket tabulated (detab).
//
// The ring holds R = D+2+kRowSlack rows (slot n % R).
#include <cuda_runtime.h>

#include "fdtd_internal.cuh"

namespace fdtd {

__device__ __forceinline__ cd ldcg(const cd* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return cd{v.x, v.y};
}
// ring rows completed before this row's wait: cached in L1 (the wait's acquire
// and fence order them before every later load of the CTA)
__device__ __forceinline__ cd ldring(const cd* p) {
  double2 v = __ldca(reinterpret_cast<const double2*>(p));
  return cd{v.x, v.y};
}
__device__ __forceinline__ cd ldro(const cd* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return cd{v.x, v.y};
}
__device__ __forceinline__ void stcg(cd* p, cd v) {
  __stcg(reinterpret_cast<double2*>(p), make_double2(v.re, v.im));
}

// psi at x = c delta <= -a, t = r delta: C phi((c-r) delta) e(r delta)
__device__ __forceinline__ cd psi_left(const MarchArgs& A, int64_t r, int64_t c) {
  const int Dh = A.D >> 1;
  cd v = ldro(&A.phitab[r - c - Dh]) * ldro(&A.etab[r]);
  if (A.phitab2) v = cfma(ldro(&A.phitab2[r - c - Dh]), ldro(&A.etab2[r]), v);  // second photon of a pair
  return A.C * v;
}

// psi at any earlier point the update of row n reads (rows n-D-1 .. n-1, or
// row n itself for columns left of -a); nslot = n % R
__device__ __forceinline__ cd psi_any(const MarchArgs& A, int64_t n, int nslot, int64_t r, int64_t c) {
  const int Dh = A.D >> 1;
  if (c <= -Dh) return psi_left(A, r, c);
  int slot = nslot - (int)(n - r);
  if (slot < 0) slot += A.R;
  return ldcg(&A.ring[(int64_t)slot * A.stride + (c + Dh - 1)]);
}

__device__ __forceinline__ cd e_theta(const MarchArgs& A, int64_t r) {
  if (r < 0) return cd{0.0, 0.0};
  cd e = ldro(&A.etab[r]);
  return (r == 0) ? 0.5 * e : e;
}

// r_m for a column of the region -a < x <= 3a (m <= 3D/2): every term read
// through psi_any.
__device__ __noinline__ cd rhs_general(const MarchArgs& A, int64_t n, int nslot, int64_t j, cd R2) {
  const int D = A.D, Dh = D >> 1;
  const int64_t m = j - Dh + 1;
  cd r = A.c1 * psi_any(A, n, nslot, n - 1, m - 1);
  r = cfma(A.c2, psi_any(A, n, nslot, n - 1, m), r);
  if (n >= D + 1) {
    cd sq = psi_any(A, n, nslot, n - D, m - D) + psi_any(A, n, nslot, n - D, m - D - 1) +
            psi_any(A, n, nslot, n - D - 1, m - D) + psi_any(A, n, nslot, n - D - 1, m - D - 1);
    r = cfma(A.c3, sq, r);
  }
  const int64_t r2 = n - m - Dh;  // line 2: t - x - a at the centre
  if (r2 >= 0) {
    double w = (r2 == 0) ? 0.5 : 1.0;
    cd bl = psi_any(A, n, nslot, r2, -m - D) + psi_any(A, n, nslot, r2, -m - D + 1);
    cd br = psi_any(A, n, nslot, r2, -m) + psi_any(A, n, nslot, r2, -m + 1);
    r = cfma(A.gs, w * (bl - br), r);
    r = cfma(R2, ldro(&A.phitab[r2]), r);  // line 4: phi((m-n) delta) = phitab[r2]
    if (A.phitab2) r = cfma(ldro(&A.rowscal2[2 * n + 1]), ldro(&A.phitab2[r2]), r);
  }
  if (m >= Dh + 1) {  // line 3, theta(x - a)
    const int64_t r3 = n - m + Dh;
    if (r3 >= 0) {
      double w = (r3 == 0) ? 0.5 : 1.0;
      cd bl = psi_any(A, n, nslot, r3, D - m) + psi_any(A, n, nslot, r3, D - m + 1);
      cd br = psi_any(A, n, nslot, r3, -m) + psi_any(A, n, nslot, r3, -m + 1);
      r = cfma(A.gs, w * (bl - br), r);
    }
  }
  return r;
}

struct RowCtx {
  int64_t n;
  int nslot;        // n % R
  const cd* row1;   // row n-1
  const cd* rowD;   // row n-D (null if n < D)
  const cd* rowD1;  // row n-D-1 (null if n < D+1)
  cd* row0;         // row n
  cd* snap;         // snapshot row or null
  cd R1, R2;
  cd R1b, R2b;      // second term of a photon pair
  cd* hs;           // shared pair sums (null: no reuse), indexed j - hbase
  int64_t hbase;
  bool cold;        // first row of this launch: pair sums not yet in shared memory
};

// r_m for x > 3a (j >= 2D), split as r_m = c2 b + q with b = psi[n-1][m]: the
// recurrence step is then y_m = c2 (y_{m-1} + b) + q, one complex product fewer.
__device__ __forceinline__ cd rhs_bulk_q(const MarchArgs& A, const RowCtx& R, int64_t j, cd& b) {
  const int D = A.D;
  cd r = A.c1 * ldring(R.row1 + j - 1);
  b = ldring(R.row1 + j);
  if (R.rowD) {
    cd hn = ldring(R.rowD + j - D - 1) + ldring(R.rowD + j - D);  // row n-D pair
    if (R.rowD1) {
      cd hp;
      if (R.hs && !R.cold) hp = R.hs[j - R.hbase];
      else hp = ldring(R.rowD1 + j - D - 1) + ldring(R.rowD1 + j - D);
      r = cfma(A.c3, hn + hp, r);
    }
    if (R.hs) R.hs[j - R.hbase] = hn;
  }
  const int64_t i = R.n - j - 1 + D;  // r2 + D
  if (i >= 0) {
    r = cfma(R.R1, ldro(&A.detab[i]), r);
    if (i >= D) r = cfma(R.R2, ldro(&A.phitab[i - D]), r);
    if (A.detab2) {
      r = cfma(R.R1b, ldro(&A.detab2[i]), r);
      if (i >= D) r = cfma(R.R2b, ldro(&A.phitab2[i - D]), r);
    }
  }
  return r;
}

__device__ __forceinline__ cd rhs_any(const MarchArgs& A, const RowCtx& R, int64_t j) {
  if (j >= 2 * (int64_t)A.D) {
    cd b;
    const cd q = rhs_bulk_q(A, R, j, b);
    return cfma(A.c2, b, q);
  }
  return rhs_general(A, R.n, R.nslot, j, R.R2);
}

// one step of the row recurrence at column j: y_j = c2 y_{j-1} + r_j
__device__ __forceinline__ cd step_any(const MarchArgs& A, const RowCtx& R, int64_t j, cd y) {
  if (j >= 2 * (int64_t)A.D) {
    cd b;
    const cd q = rhs_bulk_q(A, R, j, b);
    return cfma(A.c2, y + b, q);
  }
  return cfma(A.c2, y, rhs_general(A, R.n, R.nslot, j, R.R2));
}

// store a final value of row n and add |y|^2 to the norm (the trapezoid's
// half weight at the last column is applied once, by the CTA that owns it)
__device__ __forceinline__ void finalize(const RowCtx& R, int64_t j, cd y, double& nacc) {
  stcg(R.row0 + j, y);
  if (R.snap) stcg(R.snap + j, y);
  nacc = fma(y.re, y.re, nacc);
  nacc = fma(y.im, y.im, nacc);
}

__global__ void __launch_bounds__(kMarchThreads, 1) k_march_f64(const MarchArgs A) {
  constexpr int P = kMarchP;
  extern __shared__ cd s_h[];  // pair sums, khalo + CTA range entries
  __shared__ cd s_last[kMarchThreads];
  __shared__ int s_len[kMarchThreads];
  __shared__ cd s_carry;
  __shared__ cd s_halo[kMaxTrunc];
  __shared__ double s_red[kMarchThreads / 32];
  __shared__ int s_ok;

  const int tid = threadIdx.x;
  const int D = A.D, Dh = D >> 1;
  const int64_t j_lo = A.colsplit[blockIdx.x], j_hi = A.colsplit[blockIdx.x + 1];
  // This thread's segment [s0, s1).  A CTA inside x > 3a splits its range into
  // equal odd-length segments (the 16-byte pair sums of the 8 threads of a
  // shared-memory phase then fall in distinct banks).  A CTA that holds
  // columns of -a < x <= 3a splits by cost instead, a column there counting
  // mid_weight columns of the bulk, so that no thread is left with most of it.
  const int64_t G2 = (2 * (int64_t)D < A.nx) ? 2 * (int64_t)D : A.nx;
  int64_t s0, s1;
  if (j_lo >= G2) {
    // odd lengths; warp 0, which also waits on the neighbours and forms the halo carry,
    // takes 2 columns fewer
    const int64_t len = j_hi - j_lo;
    int64_t seg = ((len + 64 + kMarchThreads - 1) / kMarchThreads) | 1;
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
    s0 = inv(W0 + (W1 - W0) * tid / kMarchThreads);
    s1 = inv(W0 + (W1 - W0) * (tid + 1) / kMarchThreads);
  }
  const int64_t h0 = (j_lo - A.khalo > 0) ? j_lo - A.khalo : 0;  // first halo column
  const int nh = (int)(j_lo - h0);
  s_len[tid] = (int)(s1 - s0);
  __syncthreads();

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
    // the rows this CTA reads are complete and the ring slot of row n is free
    if (tid < 32) {
      const bool ok = row_wait_warp(A.deps, A.sync, A.spin_cycles, A.n_begin, blockIdx.x, n, kRowSlack);
      if (tid == 0) s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_ok) return;

    RowCtx R;
    R.n = n;
    // ring slots and the snapshot row from running counters (no 64-bit division per row)
    auto back = [&](int k) { const int t = slot - k; return t < 0 ? t + A.R : t; };
    R.nslot = slot;
    R.row1 = A.ring + (int64_t)back(1) * A.stride;
    R.rowD = (n >= D) ? A.ring + (int64_t)back(D) * A.stride : nullptr;
    R.rowD1 = (n >= D + 1) ? A.ring + (int64_t)back(D + 1) * A.stride : nullptr;
    R.row0 = A.ring + (int64_t)slot * A.stride;
    R.snap = (snap_ctr == 0) ? A.snaps + snap_idx * A.nx : nullptr;
    R.R1 = ldro(&A.rowscal[2 * n]);
    R.R2 = ldro(&A.rowscal[2 * n + 1]);
    R.R1b = A.rowscal2 ? ldro(&A.rowscal2[2 * n]) : cd{0.0, 0.0};
    R.R2b = A.rowscal2 ? ldro(&A.rowscal2[2 * n + 1]) : cd{0.0, 0.0};
    R.hs = A.hreuse ? s_h : nullptr;
    R.hbase = h0;
    R.cold = (n == A.n_begin);

    // carry into column j_lo: the true psi[n][j_lo - 1]
    if (tid < 32 && j_lo < j_hi) {
      for (int c = tid; c < nh; c += 32) s_halo[c] = rhs_any(A, R, h0 + c);
      __syncwarp();
      if (tid == 0) {
        cd y = (h0 == 0) ? psi_left(A, n, -Dh) : cd{0.0, 0.0};
        for (int c = 0; c < nh; ++c) y = cfma(A.c2, y, s_halo[c]);
        s_carry = y;
      }
    }

    // pass A: the segment from a zero carry
    double nacc = 0.0;
    cd y0[P];
    cd y = cd{0.0, 0.0};
#pragma unroll
    for (int v = 0; v < P; ++v) {
      const int64_t j = s0 + v;
      if (j < s1) y = step_any(A, R, j, y);
      y0[v] = y;
    }
    for (int64_t j = s0 + P; j < s1; ++j) {
      y = step_any(A, R, j, y);
      if (j - s0 < A.kfix) stcg(R.row0 + j, y);  // provisional: receives the carry in pass B
      else finalize(R, j, y, nacc);
    }
    s_last[tid] = (s0 < s1) ? y : cd{0.0, 0.0};
    __syncthreads();

    // pass B: carry from the threads before, added to the first kfix columns.
    // The true last value of thread u is b_u + c2^len_u (carry into u); unrolled
    // back until the product of the c2^len factors drops below 2^-60.
    if (s0 < s1) {
      cd carry = cd{0.0, 0.0}, ap = cd{1.0, 0.0};
      for (int s = 1; s <= tid + 1; ++s) {
        if (tid - s >= 0) {
          carry = cfma(ap, s_last[tid - s], carry);
          const int lu = s_len[tid - s];
          ap = ap * ((lu <= kMaxTrunc) ? A.c2pow[lu] : cd{0.0, 0.0});
          if (cabs2(ap) < 7.5e-37) break;  // (2^-60)^2
        } else {
          carry = cfma(ap, s_carry, carry);
        }
      }
#pragma unroll
      for (int v = 0; v < P; ++v) {
        const int64_t j = s0 + v;
        if (j < s1) {
          cd yv = (v < A.kfix) ? cfma(A.c2pow[v + 1], carry, y0[v]) : y0[v];
          finalize(R, j, yv, nacc);
        }
      }
      for (int v = P; v < A.kfix && s0 + v < s1; ++v) {
        const int64_t j = s0 + v;
        cd yv = cfma(A.c2pow[v + 1], carry, ldcg(R.row0 + j));
        finalize(R, j, yv, nacc);
      }
    }

    // deterministic norm partial of this CTA
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nacc += __shfl_down_sync(0xffffffffu, nacc, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = nacc;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kMarchThreads / 32; ++w) t += s_red[w];
      if (j_hi == A.nx && j_lo < j_hi) t -= 0.5 * cabs2(ldcg(R.row0 + A.nx - 1));  // trapezoid end weight
      A.partials[(n - A.n_begin) * gridDim.x + blockIdx.x] = t;
    }
    // probes of row n in this CTA's columns (its stores of row n are complete)
    if (A.probe_off && tid < 32) {
      const int k1 = A.probe_off[n + 1];
      for (int k = A.probe_off[n] + tid; k < k1; k += 32) {
        const int j = A.probe_col[k];
        if (j >= j_lo && j < j_hi) {
          const cd v = ldcg(R.row0 + j);
          A.probe_val[A.probe_idx[k]] = make_double2(v.re, v.im);
        }
      }
    }
    __syncthreads();  // row n's stores (and probes) of this CTA are issued
    if (tid == 0) {
      __threadfence();
      st_release_u64(&A.deps.done[blockIdx.x], (unsigned long long)(n + 1));
    }
  }
}

int march_f64_max_grid(int device) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march_f64, kMarchThreads, 0);
  return sms * (per > 0 ? per : 0);
}

cudaError_t launch_march_f64(const MarchArgs& a, int grid, size_t smem, cudaStream_t s) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_march_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  void* args[] = {const_cast<MarchArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)k_march_f64, dim3(grid), dim3(kMarchThreads), args, smem, s);
}

}  // namespace fdtd
