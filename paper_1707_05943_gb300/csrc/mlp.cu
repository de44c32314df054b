// mlp.cu -- BF16 tensor-core kernels of the surrogate network: a multilayer
// perceptron inputs -> GELU hidden layers -> linear outputs, trained with Adam
// on FP32 master weights.  GEMMs run on the tensor cores with mma.sync
// m16n8k16 (BF16 operands, FP32 accumulation) from shared-memory tiles; the
// first layer (4 inputs) and the element-wise steps run on the CUDA cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "fdtd_internal.cuh"

namespace fdtd {

// ---- GEMM: C[M,N] = sum_k A(m,k) B(k,n) --------------------------------------
// A(m,k) = A[m*lda + k] (ta = 0) or A[k*lda + m] (ta = 1); B(k,n) = B[n*ldb + k]
// (tb = 0) or B[k*ldb + n] (tb = 1).  M, N multiples of 64, K of 32.
enum Epi { EPI_GELU = 0, EPI_LINEAR = 1, EPI_DGELU = 2, EPI_F32 = 3 };

struct GemmArgs {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  int M, N, K, lda, ldb, ta, tb;
  int epi;
  const float* bias;        // EPI_GELU / EPI_LINEAR: bias[n]
  float* out_f32;           // EPI_GELU: pre-activation z; EPI_LINEAR / EPI_F32: result
  __nv_bfloat16* out_bf16;  // EPI_GELU: gelu(z); EPI_DGELU: acc * gelu'(zprev)
  const float* zprev;       // EPI_DGELU: pre-activation of the layer below [M,N]
  int ldo;
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float dgelu(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__global__ void __launch_bounds__(128) k_gemm_bf16(const GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 As[GBM][GBK + GPAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[GBN][GBK + GPAD];  // [n][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // warp tile 32 x 32
  const int gid = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

  for (int k0 = 0; k0 < g.K; k0 += GBK) {
    // tiles into shared memory, reading along the contiguous global dimension
    for (int idx = tid; idx < GBM * GBK; idx += 128) {
      int m, k;
      if (!g.ta) { m = idx / GBK; k = idx % GBK; }
      else { k = idx / GBM; m = idx % GBM; }
      As[m][k] = g.ta ? g.A[(size_t)(k0 + k) * g.lda + (m0 + m)] : g.A[(size_t)(m0 + m) * g.lda + (k0 + k)];
      int n, kk;
      if (!g.tb) { n = idx / GBK; kk = idx % GBK; }
      else { kk = idx / GBN; n = idx % GBN; }
      Bs[n][kk] = g.tb ? g.B[(size_t)(k0 + kk) * g.ldb + (n0 + n)] : g.B[(size_t)(n0 + n) * g.ldb + (k0 + kk)];
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GBK; ks += 16) {
      unsigned a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + gid;
        a[i][0] = *reinterpret_cast<const unsigned*>(&As[r][ks + 2 * tig]);
        a[i][1] = *reinterpret_cast<const unsigned*>(&As[r + 8][ks + 2 * tig]);
        a[i][2] = *reinterpret_cast<const unsigned*>(&As[r][ks + 2 * tig + 8]);
        a[i][3] = *reinterpret_cast<const unsigned*>(&As[r + 8][ks + 2 * tig + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + j * 8 + gid;
        b[j][0] = *reinterpret_cast<const unsigned*>(&Bs[c][ks + 2 * tig]);
        b[j][1] = *reinterpret_cast<const unsigned*>(&Bs[c][ks + 2 * tig + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]), "r"(b[j][1]));
    }
    __syncthreads();
  }
  // epilogue: accumulator element (row gid / gid+8, cols 2 tig, 2 tig + 1)
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm + i * 16 + gid + ((r >= 2) ? 8 : 0);
        const int n = n0 + wn + j * 8 + 2 * tig + (r & 1);
        const size_t o = (size_t)m * g.ldo + n;
        float v = acc[i][j][r];
        if (g.epi == EPI_GELU) {
          v += g.bias[n];
          g.out_f32[o] = v;
          g.out_bf16[o] = __float2bfloat16(gelu(v));
        } else if (g.epi == EPI_LINEAR) {
          g.out_f32[o] = v + g.bias[n];
        } else if (g.epi == EPI_DGELU) {
          g.out_bf16[o] = __float2bfloat16(v * dgelu(g.zprev[o]));
        } else {
          g.out_f32[o] = v;
        }
      }
}

// first layer: z[b,n] = sum_k x[b,k] W[n,k] + bias[n] (K = in_dim, tiny), FP32
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
// mean-squared error: dy = 2 (y - t) / (B N), loss accumulated in FP32 per block
__global__ void k_mse(const float* y, const float* t, int total, float scale, __nv_bfloat16* dy, float* dy32,
                      float* loss) {
  __shared__ float red[256];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  float d = 0.f, l = 0.f;
  if (i < total) {
    d = y[i] - t[i];
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
__global__ void k_bias_grad_f32(const float* dz, int B, int N, float* db) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dz[b * N + n];
  db[n] = s;
}
// Adam on FP32 masters; BF16 copies of the weights refreshed
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

static cudaError_t gemm(const GemmArgs& g, cudaStream_t s) {
  dim3 grid(g.N / GBN, g.M / GBM);
  k_gemm_bf16<<<grid, 128, 0, s>>>(g);
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

fdtd_status check(const fdtd_mlp* d, int batch) {
  if (!d || d->struct_size != sizeof(fdtd_mlp) || d->n_layers < 2 || d->n_layers > 7) return FDTD_ERR_INVALID_ARG;
  if (batch <= 0 || batch % 64) return FDTD_ERR_INVALID_ARG;
  for (int l = 1; l <= d->n_layers; ++l)
    if (d->dims[l] <= 0 || d->dims[l] % 64) return FDTD_ERR_INVALID_ARG;
  if (d->dims[0] <= 0 || d->dims[0] > 64) return FDTD_ERR_INVALID_ARG;
  if (!d->params || !d->params_bf16) return FDTD_ERR_INVALID_ARG;
  return FDTD_OK;
}

// workspace: per layer z (FP32) and a (BF16) of [batch, width]; output y; dy (bf16, f32); dz buffers
struct Ws {
  float* z[8];
  __nv_bfloat16* a[8];
  float* y;
  __nv_bfloat16* dz[2];
  float* dy32;
};
size_t ws_layout(const fdtd_mlp* d, int batch, char* base, Ws* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += (bytes + 255) / 256 * 256;
    return p;
  };
  int maxw = 0;
  for (int l = 1; l <= d->n_layers; ++l) maxw = maxw > d->dims[l] ? maxw : d->dims[l];
  for (int l = 0; l < d->n_layers - 1; ++l) {
    w->z[l] = (float*)take(sizeof(float) * (size_t)batch * d->dims[l + 1]);
    w->a[l] = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * (size_t)batch * d->dims[l + 1]);
  }
  w->y = (float*)take(sizeof(float) * (size_t)batch * d->dims[d->n_layers]);
  w->dz[0] = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * (size_t)batch * maxw);
  w->dz[1] = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * (size_t)batch * maxw);
  w->dy32 = (float*)take(sizeof(float) * (size_t)batch * d->dims[d->n_layers]);
  return off;
}

cudaError_t forward(const fdtd_mlp* d, const float* x, int batch, const Ws& w, cudaStream_t s) {
  int64_t offW[8], offb[8], total;
  layer_offsets(d, offW, offb, &total);
  const __nv_bfloat16* wb = static_cast<const __nv_bfloat16*>(d->params_bf16);
  const int N0 = d->dims[1], K0 = d->dims[0];
  k_layer0_fwd<<<(batch * N0 + 255) / 256, 256, 0, s>>>(x, d->params + offW[0], d->params + offb[0], batch, K0, N0,
                                                        w.z[0], w.a[0]);
  for (int l = 1; l < d->n_layers; ++l) {
    GemmArgs g = {};
    g.A = w.a[l - 1];
    g.B = wb + offW[l];
    g.M = batch;
    g.N = d->dims[l + 1];
    g.K = d->dims[l];
    g.lda = d->dims[l];
    g.ldb = d->dims[l];
    g.ta = 0;
    g.tb = 0;  // B(k,n) = W[n][k]
    g.bias = d->params + offb[l];
    g.ldo = g.N;
    if (l < d->n_layers - 1) {
      g.epi = EPI_GELU;
      g.out_f32 = w.z[l];
      g.out_bf16 = w.a[l];
    } else {
      g.epi = EPI_LINEAR;
      g.out_f32 = w.y;
    }
    cudaError_t e = gemm(g, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
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
  if (st != FDTD_OK) return st;
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
  if (!x || !y || !ws) return FDTD_ERR_INVALID_ARG;
  Ws w;
  ws_layout(d, batch, static_cast<char*>(ws), &w);
  cudaStream_t s = (cudaStream_t)stream;
  if (forward(d, x, batch, w, s) != cudaSuccess) return FDTD_ERR_CUDA;
  const size_t nout = (size_t)batch * d->dims[d->n_layers];
  if (cudaMemcpyAsync(y, w.y, sizeof(float) * nout, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return FDTD_ERR_CUDA;
  return FDTD_OK;
}

fdtd_status fdtd_mlp_train_step(const fdtd_mlp* d, const float* x, const float* target, int32_t batch, float lr,
                                int32_t step, void* ws, float* loss, void* stream) {
  fdtd_status st = check(d, batch);
  if (st != FDTD_OK) return st;
  if (!x || !target || !ws || !loss || !d->grads || (lr > 0 && (!d->adam_m || !d->adam_v)) || step < 1)
    return FDTD_ERR_INVALID_ARG;
  Ws w;
  ws_layout(d, batch, static_cast<char*>(ws), &w);
  cudaStream_t s = (cudaStream_t)stream;
  if (forward(d, x, batch, w, s) != cudaSuccess) return FDTD_ERR_CUDA;
  int64_t offW[8], offb[8], total;
  layer_offsets(d, offW, offb, &total);
  const __nv_bfloat16* wb = static_cast<const __nv_bfloat16*>(d->params_bf16);
  const int L = d->n_layers, Nout = d->dims[L];
  const int tot = batch * Nout;
  cudaMemsetAsync(loss, 0, sizeof(float), s);
  k_mse<<<(tot + 255) / 256, 256, 0, s>>>(w.y, target, tot, 1.f / (float)tot, w.dz[0], w.dy32, loss);
  // output layer (linear): dW = dy^T a_{L-2}, db = sum dy
  int cur = 0;
  for (int l = L - 1; l >= 1; --l) {
    const int N = d->dims[l + 1], K = d->dims[l];
    // weight gradient: dW[n,k] = sum_b dz[b,n] a[b,k]
    GemmArgs gw = {};
    gw.A = w.dz[cur];
    gw.ta = 1;
    gw.lda = N;  // A(m=n, k=b) = dz[b*N + n]
    gw.B = w.a[l - 1];
    gw.tb = 1;
    gw.ldb = K;  // B(k=b, n=k) = a[b*K + k]
    gw.M = N;
    gw.N = K;
    gw.K = batch;
    gw.epi = EPI_F32;
    gw.out_f32 = d->grads + offW[l];
    gw.ldo = K;
    if (gemm(gw, s) != cudaSuccess) return FDTD_ERR_CUDA;
    if (l == L - 1) k_bias_grad_f32<<<(N + 127) / 128, 128, 0, s>>>(w.dy32, batch, N, d->grads + offb[l]);
    else k_bias_grad_bf16<<<(N + 127) / 128, 128, 0, s>>>(w.dz[cur], batch, N, d->grads + offb[l]);
    // data gradient through GELU of the layer below: dz_{l-1} = (dz_l W_l) * gelu'(z_{l-1})
    GemmArgs gd = {};
    gd.A = w.dz[cur];
    gd.ta = 0;
    gd.lda = N;  // A(m=b, k=n) = dz[b*N + n]
    gd.B = wb + offW[l];
    gd.tb = 1;
    gd.ldb = K;  // B(k=n, n=k) = W[n*K + k]
    gd.M = batch;
    gd.N = K;
    gd.K = N;
    gd.epi = EPI_DGELU;
    gd.zprev = w.z[l - 1];
    gd.out_bf16 = w.dz[cur ^ 1];
    gd.ldo = K;
    if (gemm(gd, s) != cudaSuccess) return FDTD_ERR_CUDA;
    cur ^= 1;
  }
  // first layer
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
                           int32_t ldb, int32_t ta, int32_t tb, void* stream) {
  if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || M % 64 || N % 64 || K % 32) return FDTD_ERR_INVALID_ARG;
  GemmArgs g = {};
  g.A = static_cast<const __nv_bfloat16*>(A);
  g.B = static_cast<const __nv_bfloat16*>(B);
  g.M = M;
  g.N = N;
  g.K = K;
  g.lda = lda;
  g.ldb = ldb;
  g.ta = ta;
  g.tb = tb;
  g.epi = EPI_F32;
  g.out_f32 = C;
  g.ldo = N;
  return gemm(g, (cudaStream_t)stream) == cudaSuccess ? FDTD_OK : FDTD_ERR_CUDA;
}

}  // extern "C"
