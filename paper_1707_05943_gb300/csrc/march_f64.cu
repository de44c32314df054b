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
// y_m = c2 y_{m-1} + r_m.  |c2| = |W delta| / |4 + W delta| < 1, so the
// influence of a carry dies as |c2|^k; the recurrence is evaluated exactly
// where that influence exceeds 2^-60 and truncated beyond.
//
// Work layout: one persistent cooperative CTA per SM; CTA b owns the columns
// [colsplit[b], colsplit[b+1]) of every row and sweeps them in chunks of
// 512 threads x 4 consecutive columns.  Inside a chunk each thread runs the
// recurrence over its 4 columns from zero, then takes its carry from the
// previous threads' last values (kscan terms), then adds c2^(v+1) carry to
// its first kfix columns.  The carry into a CTA's first column is the
// recurrence run over khalo columns to its left (or the exact boundary value
// psi(-a, t) for the first CTA).  A grid-wide barrier with a bounded wait
// separates rows: every read of row n-1, n-D and n-D-1 is then complete.
//
// Reads of x <= -a use psi(x,t) = C phi(x-t) e(t) from the boundary tables.
// Beyond x > 3a every mirror read of lines 2-3 lands in x <= -a, and the
// sources collapse to R1(n) (E(r2) - E(r3)) + R2(n) phi(r2), with
// r2 = n - m - D/2, r3 = r2 + D and E(r) = theta(r) e(r delta).
//
// The ring holds D+2 rows (slot n % (D+2)); loads of ring rows written in this
// launch bypass L1 (ld.global.cg).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fdtd_internal.cuh"

namespace fdtd {

__device__ __forceinline__ cd ldcg(const cd* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
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
  return A.C * (ldro(&A.phitab[r - c - Dh]) * ldro(&A.etab[r]));
}

// psi at any earlier point the update reads (rows n-D-1 .. n-1, or the current
// row for columns left of -a)
__device__ __forceinline__ cd psi_any(const MarchArgs& A, int64_t r, int64_t c) {
  const int Dh = A.D >> 1;
  if (c <= -Dh) return psi_left(A, r, c);
  return ldcg(&A.ring[(r % A.R) * A.stride + (c + Dh - 1)]);
}

__device__ __forceinline__ cd e_theta(const MarchArgs& A, int64_t r) {
  if (r < 0) return cd{0.0, 0.0};
  cd e = ldro(&A.etab[r]);
  return (r == 0) ? 0.5 * e : e;
}

// r_m for a column of the region -a < x <= 3a (m <= 3D/2): every term read
// through psi_any.
__device__ cd rhs_general(const MarchArgs& A, int64_t n, int64_t j, cd R2) {
  const int D = A.D, Dh = D >> 1;
  const int64_t m = j - Dh + 1;
  cd r = A.c1 * psi_any(A, n - 1, m - 1);
  r = cfma(A.c2, psi_any(A, n - 1, m), r);
  if (n >= D + 1) {
    cd sq = psi_any(A, n - D, m - D) + psi_any(A, n - D, m - D - 1) + psi_any(A, n - D - 1, m - D) +
            psi_any(A, n - D - 1, m - D - 1);
    r = cfma(A.c3, sq, r);
  }
  const int64_t r2 = n - m - Dh;  // line 2: t - x - a at the centre
  if (r2 >= 0) {
    double w = (r2 == 0) ? 0.5 : 1.0;
    cd bl = psi_any(A, r2, -m - D) + psi_any(A, r2, -m - D + 1);
    cd br = psi_any(A, r2, -m) + psi_any(A, r2, -m + 1);
    r = cfma(A.gs, w * (bl - br), r);
    r = cfma(R2, ldro(&A.phitab[r2]), r);  // line 4: phi((m-n) delta) = phitab[r2]
  }
  if (m >= Dh + 1) {  // line 3, theta(x - a)
    const int64_t r3 = n - m + Dh;
    if (r3 >= 0) {
      double w = (r3 == 0) ? 0.5 : 1.0;
      cd bl = psi_any(A, r3, D - m) + psi_any(A, r3, D - m + 1);
      cd br = psi_any(A, r3, -m) + psi_any(A, r3, -m + 1);
      r = cfma(A.gs, w * (bl - br), r);
    }
  }
  return r;
}

// r_m for x > 3a (j >= 2D).
__device__ __forceinline__ cd rhs_bulk(const MarchArgs& A, int64_t n, int64_t j, const cd* row1, const cd* rowD,
                                       const cd* rowD1, cd R1, cd R2) {
  const int D = A.D;
  cd r = A.c1 * ldcg(row1 + j - 1);
  r = cfma(A.c2, ldcg(row1 + j), r);
  if (rowD1) {
    cd sq = ldcg(rowD + j - D) + ldcg(rowD + j - D - 1) + ldcg(rowD1 + j - D) + ldcg(rowD1 + j - D - 1);
    r = cfma(A.c3, sq, r);
  }
  const int64_t r2 = n - j - 1;  // n - m - D/2 with m = j - D/2 + 1
  r = cfma(R1, e_theta(A, r2) - e_theta(A, r2 + D), r);
  if (r2 >= 0) r = cfma(R2, ldro(&A.phitab[r2]), r);
  return r;
}

__device__ __forceinline__ cd rhs_any(const MarchArgs& A, int64_t n, int64_t j, const cd* row1, const cd* rowD,
                                      const cd* rowD1, cd R1, cd R2) {
  if (j >= 2 * (int64_t)A.D) return rhs_bulk(A, n, j, row1, rowD, rowD1, R1, R2);
  return rhs_general(A, n, j, R2);
}

// Grid-wide barrier with a bounded wait.  Returns false if any CTA has
// latched an error (its own timeout included).
__device__ bool grid_barrier(SyncWords* s, long long spin_cycles, int64_t row) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &s->bar_gen;
    unsigned int my = *gen;
    __threadfence();
    unsigned int prev = atomicAdd(&s->bar_count, 1u);
    int ok = 1;
    if (prev == gridDim.x - 1) {
      atomicExch(&s->bar_count, 0u);
      __threadfence();
      atomicAdd(&s->bar_gen, 1u);
    } else {
      long long t0 = clock64();
      while (*gen == my) {
        if (clock64() - t0 > spin_cycles) {
          if (atomicCAS(&s->status, 0u, (unsigned)FDTD_ERR_TIMEOUT) == 0u) s->where = row;
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    if (*(volatile unsigned int*)&s->status != 0u) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(kMarchThreads, 1) k_march_f64(const MarchArgs A) {
  constexpr int V = kMarchV;
  __shared__ cd s_last[kMarchThreads];
  __shared__ cd s_carry;
  __shared__ cd s_halo[kMaxTrunc];
  __shared__ double s_red[kMarchThreads / 32];

  const int tid = threadIdx.x;
  const int D = A.D, Dh = D >> 1;
  const int64_t j_lo = A.colsplit[blockIdx.x], j_hi = A.colsplit[blockIdx.x + 1];
  const int64_t nx = A.nx;

  for (int64_t n = A.n_begin; n < A.n_end; ++n) {
    const cd* row1 = A.ring + ((n - 1) % A.R) * A.stride;
    const cd* rowD = (n >= D) ? A.ring + ((n - D) % A.R) * A.stride : nullptr;
    const cd* rowD1 = (n >= D + 1) ? A.ring + ((n - D - 1) % A.R) * A.stride : nullptr;
    cd* row0 = A.ring + (n % A.R) * A.stride;
    const cd R1 = ldro(&A.rowscal[2 * n]), R2 = ldro(&A.rowscal[2 * n + 1]);
    cd* snap = (A.snaps && A.tstep >= 0 && n % (A.tstep + 1) == 0) ? A.snaps + (n / (A.tstep + 1)) * nx : nullptr;

    // carry into column j_lo: the true psi[n][j_lo - 1]
    if (j_lo < j_hi) {
      const int64_t h0 = (j_lo - A.khalo > 0) ? j_lo - A.khalo : 0;
      const int nh = (int)(j_lo - h0);
      if (tid < 32) {
        for (int c = tid; c < nh; c += 32) s_halo[c] = rhs_any(A, n, h0 + c, row1, rowD, rowD1, R1, R2);
        __syncwarp();
        if (tid == 0) {
          cd y = (h0 == 0) ? psi_left(A, n, -Dh) : cd{0.0, 0.0};
          for (int c = 0; c < nh; ++c) y = cfma(A.c2, y, s_halo[c]);
          s_carry = y;
        }
      }
    }
    __syncthreads();

    double nacc = 0.0;
    for (int64_t jc = j_lo; jc < j_hi; jc += kMarchChunk) {
      const int64_t j0 = jc + (int64_t)tid * V;
      cd y[V];
      cd prev = cd{0.0, 0.0};
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int64_t j = j0 + v;
        cd r = (j < j_hi) ? rhs_any(A, n, j, row1, rowD, rowD1, R1, R2) : cd{0.0, 0.0};
        prev = cfma(A.c2, prev, r);
        y[v] = prev;
      }
      s_last[tid] = y[V - 1];
      __syncthreads();
      // carry into this thread's first column
      const cd carry0 = s_carry;
      cd carry = cd{0.0, 0.0};
      for (int s = 1; s <= A.kscan; ++s) {
        if (tid - s >= 0) {
          carry = cfma(A.Apow[s - 1], s_last[tid - s], carry);
        } else {
          carry = cfma(A.Apow[s - 1], carry0, carry);
          break;
        }
      }
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (v < A.kfix) y[v] = cfma(A.c2pow[v + 1], carry, y[v]);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int64_t j = j0 + v;
        if (j < j_hi) {
          stcg(row0 + j, y[v]);
          if (snap) stcg(snap + j, y[v]);
          double p2 = cabs2(y[v]);
          nacc += (j == nx - 1) ? 0.5 * p2 : p2;
        }
      }
      __syncthreads();  // all threads have read s_carry / s_last
      const int64_t jlast = ((jc + kMarchChunk < j_hi) ? jc + kMarchChunk : j_hi) - 1;
      if (jlast >= j0 && jlast < j0 + V) {
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (j0 + v == jlast) s_carry = y[v];
      }
      __syncthreads();
    }

    // deterministic norm partial of this CTA
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nacc += __shfl_down_sync(0xffffffffu, nacc, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = nacc;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kMarchThreads / 32; ++w) t += s_red[w];
      A.partials[(n & 1) * gridDim.x + blockIdx.x] = t;
    }
    if (!grid_barrier(A.sync, A.spin_cycles, n)) return;
    if (blockIdx.x == 0 && tid == 0) {
      const double* pp = A.partials + (n & 1) * gridDim.x;
      double t = 0.5 * cabs2(psi_left(A, n, -Dh));
      for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(pp + b);
      A.norms[n] = A.delta * t;
    }
  }
}

int march_f64_max_grid(int device) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march_f64, kMarchThreads, 0);
  return sms * (per > 0 ? per : 0);
}

cudaError_t launch_march_f64(const MarchArgs& a, int grid, cudaStream_t s) {
  void* args[] = {const_cast<MarchArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)k_march_f64, dim3(grid), dim3(kMarchThreads), args, 0, s);
}

}  // namespace fdtd
