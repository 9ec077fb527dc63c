// fv_mlp.cu -- training and batch inference of the learned face-flux
// correction network (16 -> 64 -> 64 -> 4, GELU) on the tensor cores: every
// matrix product is a BF16 x BF16 -> FP32 mma.sync GEMM, split along K with
// fixed chunks and reduced in a fixed order (deterministic); activations,
// loss gradient, column sums and Adam are elementwise kernels.
//
// Forward (batch B):  Z1 = X W1^T + b1, H1 = gelu(Z1), Z2 = H1 W2^T + b2,
//                     H2 = gelu(Z2), Y = H2 W3^T + b3;  L = mean((Y - T)^2).
// Backward:           dY = 2 (Y - T) / (4B); dW3 = dY^T H2; db3 = 1^T dY;
//                     dZ2 = (dY W3) . gelu'(Z2); dW2 = dZ2^T H1; db2 = 1^T dZ2;
//                     dZ1 = (dZ2 W2) . gelu'(Z1); dW1 = dZ1^T X; db1 = 1^T dZ1.
// Weights and activations enter the products rounded to BF16; the master
// parameters, Z, gradients and Adam moments stay FP32.
#include <stdio.h>

#include <new>

#include "fv_internal.h"
#include "fv_mma.cuh"

namespace fv {

// ---------------------------------------------------------------------------
// GEMM: part[s][m][n] = sum_{k in chunk s} A(m,k) B(k,n), one warp per 16x8
// output tile and K chunk; A(m,k) = A[m sam + k sak], B(k,n) = B[k sbk + n sbn]
// (bf16 bits), zero outside [0,M) x [0,K) x [0,N).
// ---------------------------------------------------------------------------
struct GemmArgs {
  const uint16_t* A;
  int64_t sam, sak;
  const uint16_t* B;
  int64_t sbk, sbn;
  int64_t M, N, K, kchunk;
  int splits;
  float* part;
};

__device__ __forceinline__ uint16_t ld_bf16(const uint16_t* p, bool ok) {
  return ok ? __ldg(p) : (uint16_t)0;
}

__global__ void __launch_bounds__(128) gemm_kernel(GemmArgs g) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  const int64_t tm_n = (g.M + 15) / 16, tn_n = (g.N + 7) / 8;
  const int64_t tiles = tm_n * tn_n;
  if (warp >= tiles * g.splits) return;
  const int split = (int)(warp / tiles);
  const int64_t tile = warp - (int64_t)split * tiles;
  const int64_t m0 = (tile / tn_n) * 16, n0 = (tile % tn_n) * 8;
  const int gi = lane >> 2, ti = lane & 3;
  const int64_t k_lo = (int64_t)split * g.kchunk;
  const int64_t k_hi = k_lo + g.kchunk < g.K ? k_lo + g.kchunk : g.K;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  const int64_t ma = m0 + gi, mb = m0 + gi + 8, nb = n0 + gi;
  for (int64_t k0 = k_lo; k0 < k_hi; k0 += 16) {
    const int64_t ka = k0 + 2 * ti, kb = k0 + 2 * ti + 8;
    uint32_t a[4], b[2];
    a[0] = pack_bf16_raw(ld_bf16(g.A + ma * g.sam + ka * g.sak, ma < g.M && ka < k_hi),
                         ld_bf16(g.A + ma * g.sam + (ka + 1) * g.sak, ma < g.M && ka + 1 < k_hi));
    a[1] = pack_bf16_raw(ld_bf16(g.A + mb * g.sam + ka * g.sak, mb < g.M && ka < k_hi),
                         ld_bf16(g.A + mb * g.sam + (ka + 1) * g.sak, mb < g.M && ka + 1 < k_hi));
    a[2] = pack_bf16_raw(ld_bf16(g.A + ma * g.sam + kb * g.sak, ma < g.M && kb < k_hi),
                         ld_bf16(g.A + ma * g.sam + (kb + 1) * g.sak, ma < g.M && kb + 1 < k_hi));
    a[3] = pack_bf16_raw(ld_bf16(g.A + mb * g.sam + kb * g.sak, mb < g.M && kb < k_hi),
                         ld_bf16(g.A + mb * g.sam + (kb + 1) * g.sak, mb < g.M && kb + 1 < k_hi));
    b[0] = pack_bf16_raw(ld_bf16(g.B + ka * g.sbk + nb * g.sbn, nb < g.N && ka < k_hi),
                         ld_bf16(g.B + (ka + 1) * g.sbk + nb * g.sbn, nb < g.N && ka + 1 < k_hi));
    b[1] = pack_bf16_raw(ld_bf16(g.B + kb * g.sbk + nb * g.sbn, nb < g.N && kb < k_hi),
                         ld_bf16(g.B + (kb + 1) * g.sbk + nb * g.sbn, nb < g.N && kb + 1 < k_hi));
    mma_16816(acc, a, b);
  }
  float* out = g.part + (int64_t)split * g.M * g.N;
  const int64_t nc = n0 + 2 * ti;
  if (ma < g.M) {
    if (nc < g.N) out[ma * g.N + nc] = acc[0];
    if (nc + 1 < g.N) out[ma * g.N + nc + 1] = acc[1];
  }
  if (mb < g.M) {
    if (nc < g.N) out[mb * g.N + nc] = acc[2];
    if (nc + 1 < g.N) out[mb * g.N + nc + 1] = acc[3];
  }
}

// out[e] = sum over splits (fixed order) + bias[e % N]
__global__ void gemm_reduce_kernel(const float* __restrict__ part, int splits, int64_t MN,
                                   int64_t N, const float* __restrict__ bias, float* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MN;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += part[(int64_t)k * MN + e];
    out[e] = bias ? s + bias[e % N] : s;
  }
}

static int blocks_for(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

// C (M x N, fp32) = A B (+ bias), split along K in chunks of kchunk.
static cudaError_t gemm(cudaStream_t st, const uint16_t* A, int64_t sam, int64_t sak,
                        const uint16_t* B, int64_t sbk, int64_t sbn, int64_t M, int64_t N,
                        int64_t K, int64_t kchunk, float* part, const float* bias, float* C) {
  GemmArgs g;
  g.A = A;
  g.sam = sam;
  g.sak = sak;
  g.B = B;
  g.sbk = sbk;
  g.sbn = sbn;
  g.M = M;
  g.N = N;
  g.K = K;
  g.kchunk = kchunk;
  g.splits = (int)((K + kchunk - 1) / kchunk);
  g.part = part;
  const int64_t warps = ((M + 15) / 16) * ((N + 7) / 8) * g.splits;
  gemm_kernel<<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(g);
  gemm_reduce_kernel<<<blocks_for(M * N), 256, 0, st>>>(part, g.splits, M * N, N, bias, C);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Elementwise kernels
// ---------------------------------------------------------------------------
__global__ void to_bf16_kernel(const float* __restrict__ x, int64_t n, uint16_t* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = f32_to_bf16(x[i]);
}
__global__ void fill_bf16_kernel(uint16_t* y, int64_t n, float v) {
  const uint16_t b = f32_to_bf16(v);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = b;
}
__global__ void gelu_fwd_kernel(const float* __restrict__ z, int64_t n, uint16_t* h) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    h[i] = f32_to_bf16(gelu_f(z[i]));
}
__global__ void gelu_bwd_kernel(const float* __restrict__ dh, const float* __restrict__ z,
                                int64_t n, uint16_t* dz) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dz[i] = f32_to_bf16(dh[i] * gelu_prime_f(z[i]));
}
// dY = scale (Y - T) as bf16; per-block partial sums of (Y - T)^2
__global__ void mse_grad_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                int64_t n, float scale, uint16_t* dy, float* partial) {
  __shared__ float red[256];
  float s = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float r = y[i] - t[i];
    s += r * r;
    dy[i] = f32_to_bf16(scale * r);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}
__global__ void loss_finish_kernel(const float* __restrict__ partial, int nb, float inv_n,
                                   float* loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < nb; ++i) s += partial[i];
    *loss = s * inv_n;
  }
}
// Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// theta -= lr mhat / (sqrt(vhat) + eps) with bias-corrected mhat, vhat.
__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* m,
                            float* v, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace fv

// ---------------------------------------------------------------------------
// Trainer: workspace for batches up to max_batch.
// ---------------------------------------------------------------------------
struct fv_mlp_trainer {
  cudaStream_t stream = nullptr;
  int64_t max_batch = 0;
  void* ws = nullptr;
  uint16_t *wb, *xb, *h1, *h2, *dy, *dz2, *dz1, *ones;
  float *z1, *z2, *y, *dh2, *dh1, *part, *grad, *m, *v, *lpart;
  int64_t part_len = 0;
};

namespace {
constexpr int64_t kChunk = 2048;  // K chunk of the batch-reduction GEMMs
constexpr int kLossBlocks = 256;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Forward pass of batch B into the workspace (weights rounded to bf16 first).
cudaError_t forward(fv_mlp_trainer* t, const float* params, const float* x, int64_t B) {
  using namespace fv;
  cudaStream_t st = t->stream;
  to_bf16_kernel<<<blocks_for(kMlpParams), 256, 0, st>>>(params, kMlpParams, t->wb);
  to_bf16_kernel<<<blocks_for(B * kMlpIn), 256, 0, st>>>(x, B * kMlpIn, t->xb);
  cudaError_t e;
  // Z1 (B x 64) = X (B x 16) W1^T: A(m,k) = xb[m*16+k], B(k,n) = W1[n*16+k]
  e = gemm(st, t->xb, kMlpIn, 1, t->wb + kOffW1, 1, kMlpIn, B, kMlpHid, kMlpIn, kMlpIn, t->part,
           params + kOffB1, t->z1);
  if (e != cudaSuccess) return e;
  gelu_fwd_kernel<<<blocks_for(B * kMlpHid), 256, 0, st>>>(t->z1, B * kMlpHid, t->h1);
  e = gemm(st, t->h1, kMlpHid, 1, t->wb + kOffW2, 1, kMlpHid, B, kMlpHid, kMlpHid, kMlpHid,
           t->part, params + kOffB2, t->z2);
  if (e != cudaSuccess) return e;
  gelu_fwd_kernel<<<blocks_for(B * kMlpHid), 256, 0, st>>>(t->z2, B * kMlpHid, t->h2);
  return gemm(st, t->h2, kMlpHid, 1, t->wb + kOffW3, 1, kMlpHid, B, kMlpOut, kMlpHid, kMlpHid,
              t->part, params + kOffB3, t->y);
}

// Loss and gradient of the batch after forward().
cudaError_t backward(fv_mlp_trainer* t, const float* target, int64_t B, float* grad,
                     float* loss) {
  using namespace fv;
  cudaStream_t st = t->stream;
  const int64_t ny = B * kMlpOut;
  mse_grad_kernel<<<kLossBlocks, 256, 0, st>>>(t->y, target, ny, 2.0f / (float)ny, t->dy,
                                               t->lpart);
  loss_finish_kernel<<<1, 32, 0, st>>>(t->lpart, kLossBlocks, 1.0f / (float)ny, loss);
  cudaError_t e;
  // dW3 (4 x 64) = dY^T H2: A(m,k) = dy[k*4+m], B(k,n) = h2[k*64+n]
  e = gemm(st, t->dy, 1, kMlpOut, t->h2, kMlpHid, 1, kMlpOut, kMlpHid, B, kChunk, t->part,
           nullptr, grad + kOffW3);
  if (e != cudaSuccess) return e;
  // db3 = 1^T dY: A(m,k) = ones[k], B(k,n) = dy[k*4+n]
  e = gemm(st, t->ones, 0, 1, t->dy, kMlpOut, 1, 1, kMlpOut, B, kChunk, t->part, nullptr,
           grad + kOffB3);
  if (e != cudaSuccess) return e;
  // dH2 (B x 64) = dY W3: A(m,k) = dy[m*4+k], B(k,n) = W3[k*64+n]
  e = gemm(st, t->dy, kMlpOut, 1, t->wb + kOffW3, kMlpHid, 1, B, kMlpHid, kMlpOut, kMlpOut,
           t->part, nullptr, t->dh2);
  if (e != cudaSuccess) return e;
  gelu_bwd_kernel<<<blocks_for(B * kMlpHid), 256, 0, st>>>(t->dh2, t->z2, B * kMlpHid, t->dz2);
  e = gemm(st, t->dz2, 1, kMlpHid, t->h1, kMlpHid, 1, kMlpHid, kMlpHid, B, kChunk, t->part,
           nullptr, grad + kOffW2);
  if (e != cudaSuccess) return e;
  e = gemm(st, t->ones, 0, 1, t->dz2, kMlpHid, 1, 1, kMlpHid, B, kChunk, t->part, nullptr,
           grad + kOffB2);
  if (e != cudaSuccess) return e;
  // dH1 (B x 64) = dZ2 W2: B(k,n) = W2[k*64+n]
  e = gemm(st, t->dz2, kMlpHid, 1, t->wb + kOffW2, kMlpHid, 1, B, kMlpHid, kMlpHid, kMlpHid,
           t->part, nullptr, t->dh1);
  if (e != cudaSuccess) return e;
  gelu_bwd_kernel<<<blocks_for(B * kMlpHid), 256, 0, st>>>(t->dh1, t->z1, B * kMlpHid, t->dz1);
  // dW1 (64 x 16) = dZ1^T X
  e = gemm(st, t->dz1, 1, kMlpHid, t->xb, kMlpIn, 1, kMlpHid, kMlpIn, B, kChunk, t->part,
           nullptr, grad + kOffW1);
  if (e != cudaSuccess) return e;
  return gemm(st, t->ones, 0, 1, t->dz1, kMlpHid, 1, 1, kMlpHid, B, kChunk, t->part, nullptr,
              grad + kOffB1);
}
}  // namespace

extern "C" {

fv_status fv_mlp_trainer_create(fv_mlp_trainer** out, int64_t max_batch, void* stream) {
  if (!out || max_batch < 1 || max_batch > (1ll << 28)) return FV_ERR_INVALID_ARG;
  *out = nullptr;
  fv_mlp_trainer* t = new (std::nothrow) fv_mlp_trainer();
  if (!t) return FV_ERR_CUDA;
  t->stream = static_cast<cudaStream_t>(stream);
  t->max_batch = max_batch;
  const int64_t B = max_batch;
  const int64_t splits = (B + kChunk - 1) / kChunk;
  t->part_len = B * 64 > splits * 64 * 64 ? B * 64 : splits * 64 * 64;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align256(bytes);
    return o;
  };
  const size_t o_wb = take(2 * fv::kMlpParams), o_xb = take(2 * B * 16), o_h1 = take(2 * B * 64),
               o_h2 = take(2 * B * 64), o_dy = take(2 * B * 4), o_dz2 = take(2 * B * 64),
               o_dz1 = take(2 * B * 64), o_ones = take(2 * B), o_z1 = take(4 * B * 64),
               o_z2 = take(4 * B * 64), o_y = take(4 * B * 4), o_dh2 = take(4 * B * 64),
               o_dh1 = take(4 * B * 64), o_part = take(4 * t->part_len),
               o_grad = take(4 * fv::kMlpParams), o_m = take(4 * fv::kMlpParams),
               o_v = take(4 * fv::kMlpParams), o_lp = take(4 * kLossBlocks);
  cudaError_t e = cudaMalloc(&t->ws, off);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->ws, 0, off, t->stream);
  if (e != cudaSuccess) {
    if (t->ws) cudaFree(t->ws);
    delete t;
    return FV_ERR_CUDA;
  }
  char* w = static_cast<char*>(t->ws);
  t->wb = (uint16_t*)(w + o_wb);
  t->xb = (uint16_t*)(w + o_xb);
  t->h1 = (uint16_t*)(w + o_h1);
  t->h2 = (uint16_t*)(w + o_h2);
  t->dy = (uint16_t*)(w + o_dy);
  t->dz2 = (uint16_t*)(w + o_dz2);
  t->dz1 = (uint16_t*)(w + o_dz1);
  t->ones = (uint16_t*)(w + o_ones);
  t->z1 = (float*)(w + o_z1);
  t->z2 = (float*)(w + o_z2);
  t->y = (float*)(w + o_y);
  t->dh2 = (float*)(w + o_dh2);
  t->dh1 = (float*)(w + o_dh1);
  t->part = (float*)(w + o_part);
  t->grad = (float*)(w + o_grad);
  t->m = (float*)(w + o_m);
  t->v = (float*)(w + o_v);
  t->lpart = (float*)(w + o_lp);
  fv::fill_bf16_kernel<<<fv::blocks_for(B), 256, 0, t->stream>>>(t->ones, B, 1.0f);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
  if (e != cudaSuccess) {
    cudaFree(t->ws);
    delete t;
    return FV_ERR_CUDA;
  }
  *out = t;
  return FV_OK;
}

fv_status fv_mlp_trainer_destroy(fv_mlp_trainer* t) {
  if (!t) return FV_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(t->stream);
  cudaError_t e2 = cudaFree(t->ws);
  delete t;
  return (e == cudaSuccess && e2 == cudaSuccess) ? FV_OK : FV_ERR_CUDA;
}

fv_status fv_mlp_forward(fv_mlp_trainer* t, const float* params, const float* x, int64_t batch,
                         float* y) {
  if (!t || !params || !x || !y || batch < 1 || batch > t->max_batch) return FV_ERR_INVALID_ARG;
  cudaError_t e = forward(t, params, x, batch);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(y, t->y, sizeof(float) * 4 * batch, cudaMemcpyDeviceToDevice, t->stream);
  return e == cudaSuccess ? FV_OK : FV_ERR_CUDA;
}

fv_status fv_mlp_grad(fv_mlp_trainer* t, const float* params, const float* x,
                      const float* target, int64_t batch, float* grad, float* loss) {
  if (!t || !params || !x || !target || !grad || !loss || batch < 1 || batch > t->max_batch)
    return FV_ERR_INVALID_ARG;
  cudaError_t e = forward(t, params, x, batch);
  if (e == cudaSuccess) e = backward(t, target, batch, grad, loss);
  return e == cudaSuccess ? FV_OK : FV_ERR_CUDA;
}

fv_status fv_mlp_train_step(fv_mlp_trainer* t, float* params, const float* x, const float* target,
                            int64_t batch, float lr, int step, float* loss) {
  if (!t || !params || !x || !target || !loss || batch < 1 || batch > t->max_batch || step < 1 ||
      !(lr > 0.f))
    return FV_ERR_INVALID_ARG;
  cudaError_t e = forward(t, params, x, batch);
  if (e == cudaSuccess) e = backward(t, target, batch, t->grad, loss);
  if (e != cudaSuccess) return FV_ERR_CUDA;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  fv::adam_kernel<<<fv::blocks_for(fv::kMlpParams), 256, 0, t->stream>>>(
      params, t->grad, t->m, t->v, fv::kMlpParams, lr, b1, b2, 1e-8f, c1, c2);
  e = cudaGetLastError();
  return e == cudaSuccess ? FV_OK : FV_ERR_CUDA;
}

}  // extern "C"
