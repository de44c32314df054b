// mlp.cu -- kernels of the surrogate network: a multilayer perceptron
// inputs -> GELU hidden layers -> linear outputs, trained with Adam on FP32
// master weights.
//
// GEMMs run on the fifth-generation tensor cores: every product is cast as
// C[m][n] = sum_k A[m][k] B[n][k] with both operands K-contiguous BF16 in
// global memory.  A CTA owns a 128 x 128 tile of C; TMA copies 128 x 64
// slices of A and B (three stages, 128-byte swizzle) into shared memory; one
// thread issues tcgen05.mma kind::f16 (M 128, N 128, K 16 per instruction)
// into an FP32 accumulator in tensor memory, with full/empty mbarriers per
// stage; the epilogue reads the accumulator back with tcgen05.ld (thread =
// row) and fuses bias, GELU, GELU' and the BF16 casts, writing transposed
// copies where backpropagation needs the other operand order.  Layer 0 (a
// handful of inputs) and the element-wise steps run on the CUDA cores.
#include <cuda.h>  // CUtensorMap and its enums (types only; the encoder comes from the runtime)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "fdtd_internal.cuh"

namespace fdtd {

__device__ int g_mlp_status;  // 1: an mbarrier wait of the GEMM ran out

enum Epi { EPI_GELU = 0, EPI_LINEAR = 1, EPI_DGELU = 2, EPI_F32 = 3, EPI_ATOMIC = 4 };

struct NtArgs {
  const __nv_bfloat16* A;  // [M][lda], K contiguous
  const __nv_bfloat16* B;  // [N][ldb], K contiguous
  int M, N, K, lda, ldb;
  int epi;
  const float* bias;          // EPI_GELU / EPI_LINEAR: bias[n]
  float* out_f32;             // EPI_GELU: pre-activation; EPI_LINEAR / EPI_F32: result   [M][ldo]
  __nv_bfloat16* out_bf16;    // EPI_GELU: gelu(z); EPI_DGELU: acc * gelu'(zprev)        [M][ldo]
  __nv_bfloat16* out_bf16_t;  // optional transposed copy of out_bf16                     [N][ldt]
  const float* zprev;         // EPI_DGELU: [M][ldo]
  int ldo, ldt;
  int kt_split;               // K slices per split (blockIdx.z); EPI_ATOMIC adds the partial sums
  long long spin;             // clock cycles an mbarrier wait may take before giving up
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float dgelu(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

constexpr int TM = 128, TN = 128, TK = 64;
constexpr int kTileBytes = TM * TK * 2;                       // 16 KB per operand slice
constexpr uint32_t kTmemCols = TN;                            // FP32 accumulator columns
// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at 24-28
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }


__device__ __forceinline__ bool mbar_done(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false when the limit ran out
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, long long spin) {
  const long long t0 = clock64();
  while (!mbar_done(a, parity))
    if (clock64() - t0 > spin) return false;
  return true;
}

#define TC_LD32(taddr, v)                                                                                            \
  asm volatile(                                                                                                      \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19," \
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"                                                   \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),  \
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),       \
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),      \
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])                    \
      : "r"(taddr))

// epilogue: thread (warp w, lane l) owns row m0 + 32 w + l of the tile and reads its
// accumulator row from tensor memory 32 columns at a time
__device__ __forceinline__ void tc_epilogue(const NtArgs& g, uint32_t tmem, int m0, int n0, int warp, int lane) {
  const int m = m0 + warp * 32 + lane;
#pragma unroll 1
  for (int cb = 0; cb < TN; cb += 32) {
    uint32_t v[32];
    TC_LD32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    const int nb = n0 + cb;
    if (nb >= g.N || m >= g.M) continue;
    float f[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(v[j]);
    const size_t o = (size_t)m * g.ldo + nb;
    if (g.epi == EPI_GELU || g.epi == EPI_LINEAR) {
#pragma unroll
      for (int j = 0; j < 32; ++j) f[j] += __ldg(g.bias + nb + j);
    }
    if (g.epi == EPI_ATOMIC) {
#pragma unroll
      for (int j = 0; j < 32; ++j) atomicAdd(g.out_f32 + o + j, f[j]);
      continue;
    }
    if (g.epi == EPI_GELU || g.epi == EPI_LINEAR || g.epi == EPI_F32) {
#pragma unroll
      for (int j = 0; j < 32; j += 4)
        *reinterpret_cast<float4*>(g.out_f32 + o + j) = make_float4(f[j], f[j + 1], f[j + 2], f[j + 3]);
    }
    if (g.epi == EPI_GELU || g.epi == EPI_DGELU) {
      if (g.epi == EPI_GELU) {
#pragma unroll
        for (int j = 0; j < 32; ++j) f[j] = gelu(f[j]);
      } else {
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          const float4 z = *reinterpret_cast<const float4*>(g.zprev + o + j);
          f[j] *= dgelu(z.x);
          f[j + 1] *= dgelu(z.y);
          f[j + 2] *= dgelu(z.z);
          f[j + 3] *= dgelu(z.w);
        }
      }
      __align__(16) __nv_bfloat16 h[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) h[j] = __float2bfloat16(f[j]);
#pragma unroll
      for (int j = 0; j < 32; j += 8)
        *reinterpret_cast<uint4*>(g.out_bf16 + o + j) = *reinterpret_cast<const uint4*>(h + j);
      if (g.out_bf16_t) {
#pragma unroll
        for (int j = 0; j < 32; ++j) g.out_bf16_t[(size_t)(nb + j) * g.ldt + m] = h[j];
      }
    }
  }
}

// The product, with the operand slices staged by TMA: A and B are 2-D
// tensor maps (K inner) with 128-byte swizzle, so that a 128 x 64 box lands in
// shared memory in the K-major SWIZZLE_128B layout the MMA reads (8-row groups
// 1024 B apart, each row's 128 B XOR-swizzled by the row index).  Thread 0 runs
// the pipeline: it arms a stage's "full" mbarrier with the bytes of both boxes,
// issues the two copies, and, when the stage is full, issues the four MMAs of
// the slice and commits them to the stage's "empty" mbarrier, which it waits on
// before reusing the stage.  Boxes past M, N or K are zero-filled by the copy.
constexpr int kTmaStages = 3;
constexpr int kGemmSmemTma = kTmaStages * 2 * kTileBytes + 1024;

// shared-memory descriptor of a K-major SWIZZLE_128B operand: stride between
// 8-row groups 1024 B, descriptor version 1, layout type 2 (128-byte swizzle);
// the leading offset is unused for this layout
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
          "r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

__global__ void __launch_bounds__(128) k_gemm_nt_tma(const NtArgs g, const __grid_constant__ CUtensorMap tmA,
                                                     const __grid_constant__ CUtensorMap tmB) {
  extern __shared__ unsigned char dsmem[];
  __shared__ __align__(8) uint64_t full[kTmaStages], empty[kTmaStages], drain;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  unsigned char* sbase = (unsigned char*)(((uintptr_t)dsmem + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tmem_sh)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kTmaStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&drain)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_sh = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_sh;
  const int kt0 = blockIdx.z * g.kt_split;
  const int nk = min((g.K + TK - 1) / TK - kt0, g.kt_split);

  if (tid == 0) {
    auto stage_a = [&](int kt) { return su32(sbase + (size_t)(kt % kTmaStages) * 2 * kTileBytes); };
    auto issue = [&](int kt) {
      const int s = kt % kTmaStages;
      const uint32_t sA = stage_a(kt), sB = sA + kTileBytes;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(&full[s])),
                   "r"(2 * kTileBytes)
                   : "memory");
      tma_2d(sA, &tmA, (kt0 + kt) * TK, m0, su32(&full[s]));
      tma_2d(sB, &tmB, (kt0 + kt) * TK, n0, su32(&full[s]));
    };
    int issued = 0, kt = 0;
    bool bad = false, lost_full = false;
    for (; issued < nk && issued < kTmaStages; ++issued) issue(issued);
    for (; kt < nk; ++kt) {
      const int s = kt % kTmaStages;
      const uint32_t ph = (uint32_t)((kt / kTmaStages) & 1);
      if (!mbar_wait(su32(&full[s]), ph, g.spin)) {
        bad = lost_full = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sA = stage_a(kt), sB = sA + kTileBytes;
#pragma unroll
      for (int kk = 0; kk < TK / 16; ++kk) {
        const uint64_t da = sdesc_sw128(sA + kk * 32), db = sdesc_sw128(sB + kk * 32);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       su32(&empty[s]))
                   : "memory");
      if (issued < nk) {  // issued == kt + kTmaStages: stage s is next, once the MMAs above have read it
        if (!mbar_wait(su32(&empty[s]), ph, g.spin)) {
          bad = true;
          break;
        }
        issue(issued);
        ++issued;
      }
    }
    if (bad) {
      atomicExch(&g_mlp_status, 1);
      abort_sh = 1;
      // let the copies still in flight land before the CTA leaves (bounded)
      for (int k = lost_full ? kt : kt + 1; k < issued; ++k)
        mbar_wait(su32(&full[k % kTmaStages]), (uint32_t)((k / kTmaStages) & 1), g.spin);
    }
  }
  __syncthreads();
  if (!abort_sh) {
    // the last commit covers every MMA of this CTA
    const int s = (nk - 1) % kTmaStages;
    if (!mbar_wait(su32(&empty[s]), (uint32_t)(((nk - 1) / kTmaStages) & 1), g.spin)) {
      atomicExch(&g_mlp_status, 1);
      abort_sh = 1;
    }
  }
  __syncthreads();
  if (abort_sh && tid == 0) {
    // a wait gave up: MMAs committed earlier may still be reading the stages and
    // writing tensor memory.  One more commit (it tracks every MMA this thread
    // issued) on a spare barrier, waited on with the same bound, lets them
    // finish before the tensor memory is released and the CTA leaves.
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(&drain))
                 : "memory");
    mbar_wait(su32(&drain), 0u, g.spin);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (!abort_sh) tc_epilogue(g, tmem, m0, n0, warp, lane);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

// ---- CUDA-core kernels ----------------------------------------------------------

// first layer: z[b,n] = sum_k x[b,k] W[n,k] + bias[n] (K = inputs, tiny), FP32
__global__ void k_layer0_fwd(const float* x, const float* W, const float* bias, int B, int K, int N, float* z,
                             __nv_bfloat16* a) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * N) return;
  int b = idx / N, n = idx % N;
  float s = bias[n];
  for (int k = 0; k < K; ++k) s = fmaf(x[b * K + k], W[n * K + k], s);
  z[idx] = s;
  a[idx] = __float2bfloat16(gelu(s));
}
// dW0[n,k] = sum_b dz[b,n] x[b,k]
__global__ void k_layer0_wgrad(const __nv_bfloat16* dz, const float* x, int B, int K, int N, float* dW) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * K) return;
  int n = idx / K, k = idx % K;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s = fmaf(__bfloat162float(dz[b * N + n]), x[b * K + k], s);
  dW[idx] = s;
}
// db[n] = sum_b dz[b,n]
__global__ void k_bias_grad_bf16(const __nv_bfloat16* dz, int B, int N, float* db) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += __bfloat162float(dz[b * N + n]);
  db[n] = s;
}
__global__ void k_bias_grad_f32(const float* dz, int B, int N, float* db) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dz[b * N + n];
  db[n] = s;
}
// mean squared error: dy = 2 (y - t) / (B N) (BF16 and FP32), loss summed per block in FP32
__global__ void k_mse(const float* y, const float* t, int total, float scale, __nv_bfloat16* dy, float* dy32,
                      float* loss) {
  __shared__ float red[256];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < total) {
    const float d = y[i] - t[i];
    l = d * d;
    dy[i] = __float2bfloat16(2.f * d * scale);
    dy32[i] = 2.f * d * scale;
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] * scale);
}
// out[c][r] = in[r][c] for a rows x cols BF16 matrix, 32 x 32 tiles through shared memory
__global__ void k_transpose_bf16(const __nv_bfloat16* in, __nv_bfloat16* out, int rows, int cols) {
  __shared__ __nv_bfloat16 t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(size_t)c * rows + r] = t[threadIdx.x][i];
  }
}
// split-K finish of a data gradient: dz[b][k] = part[b][k] gelu'(z[b][k]) in BF16,
// with its transpose, 32 x 32 tiles through shared memory
__global__ void k_dgelu_finish(const float* part, const float* z, __nv_bfloat16* dz, __nv_bfloat16* dzt, int rows,
                               int cols) {
  __shared__ __nv_bfloat16 t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) {
      const size_t o = (size_t)r * cols + c;
      const __nv_bfloat16 h = __float2bfloat16(part[o] * dgelu(z[o]));
      dz[o] = h;
      t[i][threadIdx.x] = h;
    }
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dzt[(size_t)c * rows + r] = t[threadIdx.x][i];
  }
}
// Adam on FP32 masters (Kingma & Ba, bias-corrected)
__global__ void k_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}
__global__ void k_to_bf16(const float* p, __nv_bfloat16* q, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) q[i] = __float2bfloat16(p[i]);
}

// K splits for a product with few output tiles and a long K (0 or 1: none)
static int split_count(int M, int N, int K) {
  const int tiles = ((M + TM - 1) / TM) * ((N + TN - 1) / TN);
  const int kt = (K + TK - 1) / TK;
  if (tiles >= 76 || kt < 16) return 1;
  int sp = (152 + tiles - 1) / tiles;
  if (sp > kt / 8) sp = kt / 8;  // at least 8 slices per split
  return sp < 1 ? 1 : sp;
}

// launches the tiles of g; with splits > 1, g.epi must be EPI_ATOMIC into a zeroed FP32 C
// tensor map of a K-contiguous BF16 operand [rows][ld], boxes of 128 rows x 64 K,
// 128-byte swizzle, zero fill outside
static cudaError_t make_map(CUtensorMap* map, const __nv_bfloat16* base, int rows, int K, int ld) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(__nv_bfloat16)};
  const cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)TM};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides, box,
                         es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// launches the tiles of g; with splits > 1, g.epi must be EPI_ATOMIC into a zeroed FP32 C
static cudaError_t gemm_nt(NtArgs g, cudaStream_t s, int splits = 1) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_gemm_nt_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmemTma);
  });
  if (attr != cudaSuccess) return attr;
  g.spin = 2000000000LL;  // about a second at the SM clock
  const int kt = (g.K + TK - 1) / TK;
  g.kt_split = (kt + splits - 1) / splits;
  splits = (kt + g.kt_split - 1) / g.kt_split;
  alignas(64) CUtensorMap mA, mB;
  cudaError_t e = make_map(&mA, g.A, g.M, g.K, g.lda);
  if (e == cudaSuccess) e = make_map(&mB, g.B, g.N, g.K, g.ldb);
  if (e != cudaSuccess) return e;
  dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, splits);
  k_gemm_nt_tma<<<grid, 128, kGemmSmemTma, s>>>(g, mA, mB);
  return cudaGetLastError();
}

static cudaError_t transpose(const __nv_bfloat16* in, __nv_bfloat16* out, int rows, int cols, cudaStream_t s) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  k_transpose_bf16<<<grid, dim3(32, 8), 0, s>>>(in, out, rows, cols);
  return cudaGetLastError();
}

}  // namespace fdtd

using namespace fdtd;

namespace {

// parameter offsets (floats) of layer l: W then b
void layer_offsets(const fdtd_mlp* d, int64_t* offW, int64_t* offb, int64_t* total) {
  int64_t o = 0;
  for (int l = 0; l < d->n_layers; ++l) {
    offW[l] = o;
    o += (int64_t)d->dims[l + 1] * d->dims[l];
    offb[l] = o;
    o += d->dims[l + 1];
  }
  *total = o;
}

bool shape_ok(const fdtd_mlp* d) {
  if (!d || d->struct_size != sizeof(fdtd_mlp) || d->n_layers < 2 || d->n_layers > 7) return false;
  for (int l = 1; l <= d->n_layers; ++l)
    if (d->dims[l] <= 0 || d->dims[l] % 64) return false;
  return d->dims[0] > 0 && d->dims[0] <= 64;
}

fdtd_status check(const fdtd_mlp* d, int batch) {
  if (!shape_ok(d) || batch <= 0 || batch % 64) return FDTD_ERR_INVALID_ARG;
  if (!d->params || !d->params_bf16) return FDTD_ERR_INVALID_ARG;
  return FDTD_OK;
}

// workspace: per hidden layer z (FP32), a and a^T (BF16); output y; dz and dz^T
// (two of each, BF16); dy in FP32; one transposed weight matrix
struct Ws {
  float* z[8];
  __nv_bfloat16* a[8];
  __nv_bfloat16* at[8];
  float* y;
  __nv_bfloat16* dz[2];
  __nv_bfloat16* dzt[2];
  float* dy32;
  __nv_bfloat16* wt;
  float* part;  // split-K partial sums [batch][widest layer]
};
size_t ws_layout(const fdtd_mlp* d, int batch, char* base, Ws* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += (bytes + 255) / 256 * 256;
    return p;
  };
  int maxw = 0;
  size_t maxW = 0;
  for (int l = 1; l <= d->n_layers; ++l) maxw = maxw > d->dims[l] ? maxw : d->dims[l];
  for (int l = 1; l < d->n_layers; ++l) {
    const size_t e = (size_t)d->dims[l + 1] * d->dims[l];
    maxW = maxW > e ? maxW : e;
  }
  for (int l = 0; l < d->n_layers - 1; ++l) {
    w->z[l] = (float*)take(sizeof(float) * (size_t)batch * d->dims[l + 1]);
    w->a[l] = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * (size_t)batch * d->dims[l + 1]);
    w->at[l] = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * (size_t)batch * d->dims[l + 1]);
  }
  w->y = (float*)take(sizeof(float) * (size_t)batch * d->dims[d->n_layers]);
  for (int i = 0; i < 2; ++i) {
    w->dz[i] = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * (size_t)batch * maxw);
    w->dzt[i] = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * (size_t)batch * maxw);
  }
  w->dy32 = (float*)take(sizeof(float) * (size_t)batch * d->dims[d->n_layers]);
  w->wt = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * maxW);
  w->part = (float*)take(sizeof(float) * (size_t)batch * maxw);
  return off;
}

cudaError_t forward(const fdtd_mlp* d, const float* x, int batch, const Ws& w, bool keep_t, cudaStream_t s) {
  int64_t offW[8], offb[8], total;
  layer_offsets(d, offW, offb, &total);
  const __nv_bfloat16* wb = static_cast<const __nv_bfloat16*>(d->params_bf16);
  const int N0 = d->dims[1], K0 = d->dims[0];
  k_layer0_fwd<<<(batch * N0 + 255) / 256, 256, 0, s>>>(x, d->params + offW[0], d->params + offb[0], batch, K0, N0,
                                                        w.z[0], w.a[0]);
  if (keep_t) {
    cudaError_t e = transpose(w.a[0], w.at[0], batch, N0, s);
    if (e != cudaSuccess) return e;
  }
  for (int l = 1; l < d->n_layers; ++l) {
    NtArgs g = {};
    g.A = w.a[l - 1];
    g.lda = d->dims[l];
    g.B = wb + offW[l];  // W_l [n][k]
    g.ldb = d->dims[l];
    g.M = batch;
    g.N = d->dims[l + 1];
    g.K = d->dims[l];
    g.bias = d->params + offb[l];
    g.ldo = g.N;
    g.ldt = batch;
    if (l < d->n_layers - 1) {
      g.epi = EPI_GELU;
      g.out_f32 = w.z[l];
      g.out_bf16 = w.a[l];
      g.out_bf16_t = keep_t ? w.at[l] : nullptr;
    } else {
      g.epi = EPI_LINEAR;
      g.out_f32 = w.y;
    }
    cudaError_t e = gemm_nt(g, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// BF16 weight blocks of layers >= 1 start where the FP32 ones do, so their byte
// offsets are 2 * the float offsets: they must be 16-byte aligned for the tensor maps
bool weights_aligned(const fdtd_mlp* d) {
  int64_t offW[8], offb[8], total;
  layer_offsets(d, offW, offb, &total);
  if ((uintptr_t)d->params_bf16 & 15) return false;
  for (int l = 1; l < d->n_layers; ++l)
    if ((offW[l] * 2) & 15) return false;
  return true;
}

}  // namespace

extern "C" {

fdtd_status fdtd_mlp_param_count(const fdtd_mlp* d, int64_t* count) {
  if (!d || !count || d->n_layers < 2 || d->n_layers > 7) return FDTD_ERR_INVALID_ARG;
  int64_t offW[8], offb[8];
  layer_offsets(d, offW, offb, count);
  return FDTD_OK;
}

fdtd_status fdtd_mlp_workspace_bytes(const fdtd_mlp* d, int32_t batch, size_t* bytes) {
  fdtd_status st = check(d, batch);
  if (st != FDTD_OK || !bytes) return FDTD_ERR_INVALID_ARG;
  Ws w;
  *bytes = ws_layout(d, batch, nullptr, &w);
  return FDTD_OK;
}

fdtd_status fdtd_mlp_sync_bf16(const fdtd_mlp* d, void* stream) {
  int64_t n;
  if (fdtd_mlp_param_count(d, &n) != FDTD_OK || !d->params || !d->params_bf16) return FDTD_ERR_INVALID_ARG;
  k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      d->params, static_cast<__nv_bfloat16*>(d->params_bf16), n);
  return cudaGetLastError() == cudaSuccess ? FDTD_OK : FDTD_ERR_CUDA;
}

fdtd_status fdtd_mlp_forward(const fdtd_mlp* d, const float* x, int32_t batch, float* y, void* ws, void* stream) {
  fdtd_status st = check(d, batch);
  if (st != FDTD_OK) return st;
  if (!x || !y || !ws || ((uintptr_t)ws & 255) || !weights_aligned(d)) return FDTD_ERR_INVALID_ARG;
  Ws w;
  ws_layout(d, batch, static_cast<char*>(ws), &w);
  cudaStream_t s = (cudaStream_t)stream;
  if (forward(d, x, batch, w, false, s) != cudaSuccess) return FDTD_ERR_CUDA;
  const size_t nout = (size_t)batch * d->dims[d->n_layers];
  if (cudaMemcpyAsync(y, w.y, sizeof(float) * nout, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return FDTD_ERR_CUDA;
  return FDTD_OK;
}

fdtd_status fdtd_mlp_train_step(const fdtd_mlp* d, const float* x, const float* target, int32_t batch, float lr,
                                int32_t step, void* ws, float* loss, void* stream) {
  fdtd_status st = check(d, batch);
  if (st != FDTD_OK) return st;
  if (!x || !target || !ws || ((uintptr_t)ws & 255) || !loss || !d->grads ||
      (lr > 0 && (!d->adam_m || !d->adam_v)) || step < 1 || !weights_aligned(d))
    return FDTD_ERR_INVALID_ARG;
  Ws w;
  ws_layout(d, batch, static_cast<char*>(ws), &w);
  cudaStream_t s = (cudaStream_t)stream;
  if (forward(d, x, batch, w, true, s) != cudaSuccess) return FDTD_ERR_CUDA;
  int64_t offW[8], offb[8], total;
  layer_offsets(d, offW, offb, &total);
  const __nv_bfloat16* wb = static_cast<const __nv_bfloat16*>(d->params_bf16);
  const int L = d->n_layers, Nout = d->dims[L];
  const int tot = batch * Nout;
  if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return FDTD_ERR_CUDA;
  k_mse<<<(tot + 255) / 256, 256, 0, s>>>(w.y, target, tot, 1.f / (float)tot, w.dz[0], w.dy32, loss);
  if (transpose(w.dz[0], w.dzt[0], batch, Nout, s) != cudaSuccess) return FDTD_ERR_CUDA;
  int cur = 0;
  for (int l = L - 1; l >= 1; --l) {
    const int N = d->dims[l + 1], K = d->dims[l];
    // weight gradient: dW[n][k] = sum_b dz[b][n] a[b][k] = sum_b dz^T[n][b] a^T[k][b]
    NtArgs gw = {};
    gw.A = w.dzt[cur];
    gw.lda = batch;
    gw.B = w.at[l - 1];
    gw.ldb = batch;
    gw.M = N;
    gw.N = K;
    gw.K = batch;
    gw.epi = EPI_F32;
    gw.out_f32 = d->grads + offW[l];
    gw.ldo = K;
    if (gemm_nt(gw, s) != cudaSuccess) return FDTD_ERR_CUDA;
    if (l == L - 1) k_bias_grad_f32<<<(N + 127) / 128, 128, 0, s>>>(w.dy32, batch, N, d->grads + offb[l]);
    else k_bias_grad_bf16<<<(N + 127) / 128, 128, 0, s>>>(w.dz[cur], batch, N, d->grads + offb[l]);
    // data gradient through GELU of the layer below:
    // dz'[b][k] = gelu'(z[b][k]) sum_n dz[b][n] W[n][k], with W^T[k][n] as the K-contiguous operand
    if (transpose(wb + offW[l], w.wt, N, K, s) != cudaSuccess) return FDTD_ERR_CUDA;
    NtArgs gd = {};
    gd.A = w.dz[cur];
    gd.lda = N;
    gd.B = w.wt;
    gd.ldb = N;
    gd.M = batch;
    gd.N = K;
    gd.K = N;
    gd.ldo = K;
    gd.ldt = batch;
    const int sp = split_count(batch, K, N);
    if (sp > 1) {
      // long K over few tiles: partial sums in FP32, then GELU' and the casts
      if (cudaMemsetAsync(w.part, 0, sizeof(float) * (size_t)batch * K, s) != cudaSuccess) return FDTD_ERR_CUDA;
      gd.epi = EPI_ATOMIC;
      gd.out_f32 = w.part;
      if (gemm_nt(gd, s, sp) != cudaSuccess) return FDTD_ERR_CUDA;
      k_dgelu_finish<<<dim3((K + 31) / 32, (batch + 31) / 32), dim3(32, 8), 0, s>>>(w.part, w.z[l - 1], w.dz[cur ^ 1],
                                                                                    w.dzt[cur ^ 1], batch, K);
    } else {
      gd.epi = EPI_DGELU;
      gd.zprev = w.z[l - 1];
      gd.out_bf16 = w.dz[cur ^ 1];
      gd.out_bf16_t = w.dzt[cur ^ 1];
      if (gemm_nt(gd, s) != cudaSuccess) return FDTD_ERR_CUDA;
    }
    cur ^= 1;
  }
  {
    const int N = d->dims[1], K = d->dims[0];
    k_layer0_wgrad<<<(N * K + 255) / 256, 256, 0, s>>>(w.dz[cur], x, batch, K, N, d->grads + offW[0]);
    k_bias_grad_bf16<<<(N + 127) / 128, 128, 0, s>>>(w.dz[cur], batch, N, d->grads + offb[0]);
  }
  if (lr > 0) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(d->params, d->grads, d->adam_m, d->adam_v, total, lr, b1,
                                                         b2, 1e-8f, c1, c2);
    k_to_bf16<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(d->params, static_cast<__nv_bfloat16*>(d->params_bf16),
                                                              total);
  }
  return cudaGetLastError() == cudaSuccess ? FDTD_OK : FDTD_ERR_CUDA;
}

fdtd_status fdtd_gemm_bf16(const void* A, const void* B, float* C, int32_t M, int32_t N, int32_t K, int32_t lda,
                           int32_t ldb, void* stream) {
  if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || M % 64 || N % 64 || K % 32 || lda < K || ldb < K ||
      lda % 8 || ldb % 8 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || ((uintptr_t)C & 15))
    return FDTD_ERR_INVALID_ARG;
  NtArgs g = {};
  g.A = static_cast<const __nv_bfloat16*>(A);
  g.B = static_cast<const __nv_bfloat16*>(B);
  g.M = M;
  g.N = N;
  g.K = K;
  g.lda = lda;
  g.ldb = ldb;
  g.ldo = N;
  g.out_f32 = C;
  cudaStream_t s = (cudaStream_t)stream;
  const int sp = split_count(M, N, K);
  if (sp > 1) {
    if (cudaMemsetAsync(C, 0, sizeof(float) * (size_t)M * N, s) != cudaSuccess) return FDTD_ERR_CUDA;
    g.epi = EPI_ATOMIC;
  } else {
    g.epi = EPI_F32;
  }
  return gemm_nt(g, s, sp) == cudaSuccess ? FDTD_OK : FDTD_ERR_CUDA;
}

fdtd_status fdtd_mlp_status(void* stream) {
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return FDTD_ERR_CUDA;
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_mlp_status, sizeof v) != cudaSuccess) return FDTD_ERR_CUDA;
  if (v) {
    const int zero = 0;
    if (cudaMemcpyToSymbol(g_mlp_status, &zero, sizeof zero) != cudaSuccess) return FDTD_ERR_CUDA;
    return FDTD_ERR_TIMEOUT;
  }
  return FDTD_OK;
}

}  // extern "C"
