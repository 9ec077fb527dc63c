// fv_mlp.cu -- training and batch inference of the learned face-flux
// correction network (16 -> 64 -> 64 -> 4, GELU) on the 5th-generation tensor
// cores (tcgen05.mma: BF16 operands in shared memory, FP32 accumulators in
// tensor memory).  Not part of the paper: the correction is added on top of
// its Rusanov flux (Eq. 4).
//
// Forward (batch B):  Z1 = X W1^T + b1, H1 = gelu(Z1), Z2 = H1 W2^T + b2,
//                     H2 = gelu(Z2), Y = H2 W3^T + b3;  L = mean((Y - T)^2).
// Backward:           dY = 2 (Y - T) / (4B); dW3 = dY^T H2; db3 = 1^T dY;
//                     dZ2 = (dY W3) . gelu'(Z2); dW2 = dZ2^T H1; db2 = 1^T dZ2;
//                     dZ1 = (dZ2 W2) . gelu'(Z1); dW1 = dZ1^T X; db1 = 1^T dZ1.
// Weights, X, H1, H2, dY, dZ2 and dZ1 enter the products rounded to BF16; the
// accumulators, Z, the master parameters, gradients and Adam moments are FP32.
//
// One CTA of 128 threads walks tiles of 128 samples (thread t owns sample t
// of the tile, which is TMEM lane t of every accumulator).  Per tile, one
// elected thread issues the chain of products, and after each the threads
// read their rows back, apply the bias and activation and write the next
// operand:
//   Z1 = X W1^T, Z2 = H1 W2^T, Y = H2 W3^T           (forward)
//   dH2 = dY W3, dH1 = dZ2 W2 (and Z1 once more)     (backward, data)
//   GW3 += [H2 ; 1]^T dY,  GA += [dZ2 ; dZ1]^T [H1 ; X ; 1]   (weights)
// The weight gradients are sums over the samples: products with K = the
// tile's 128 samples, accumulated in tensor memory over all tiles of the
// CTA.  Their operands are the same shared-memory tiles as the forward ones,
// read transposed: a K-major tile of (sample, feature) rows is, byte for
// byte, an MN-major tile of (feature, sample), so no data is moved for the
// transposes.  Rows of ones among the operands give the bias gradients
// (column 80 of GA, row 64 of GW3).  A second kernel sums the CTAs' partial
// gradients in a fixed order and applies Adam, so results do not depend on
// timing.
#include <stdio.h>

#include <new>

#include "fv_device.cuh"
#include "fv_internal.h"
#include "fv_mma.cuh"
#include "fv_ptx.cuh"
#include "fv_tc.cuh"

namespace fv {
namespace {

// --- shared memory (bytes from the 1024-aligned dynamic base) -------------
// Three "paired" buffers of 16 groups of 8 samples, 2048 bytes a group.  In
// each group, the 8 samples' rows of a 64-wide BF16 operand take 1024 bytes
// as 8 core matrices (8 rows x 16 bytes); the second 1024 bytes hold other
// operands of the same samples, so that, read MN-major with 128-byte steps
// along the features, rows 64..127 of a product's A or B operand continue
// into them:
//   PC: [H1 (64) | X (16) | ones row (16) | dY (16) | unused]
//   PA: [dZ2 (64) | dZ1 (64)]
//   PB: [H2 (64) | ones row, zeros]
constexpr int kRows = 128;      // samples per tile: the MMA's M
constexpr int kGroup = 2048;    // bytes per 8 samples in a paired buffer
constexpr int kPC = 0, kPA = 32768, kPB = 65536;
constexpr int kXoff = 1024, kOnesC = 1280, kDYoff = 1536, kOnesB = 1024;
constexpr int kW1 = 98304;            // W1: 64 x 16, K-major
constexpr int kW2 = kW1 + 2048;       // W2: 64 x 64, K-major
constexpr int kW3 = kW2 + 8192;       // W3: 16 x 64 (rows 4..15 zero), K-major
constexpr int kBias = kW3 + 2048;     // b1 (64), b2 (64), b3 (4) as floats
constexpr int kSmemBytes = kBias + 132 * 4;
// --- tensor memory columns -----------------------------------------------
// W: Z1, Y, dH2 and Z1 again; Z2: Z2, then dH1; G3: dW3^T (rows 0..63) and
// db3 (row 64); GA: dW2 (rows 0..63, columns 0..63), dW1 (rows 64..127,
// columns 64..79), db2 / db1 (column 80).  Every accumulator starts at a
// multiple of 32 columns.
constexpr int kColW = 0, kColZ2 = 64, kColG3 = 128, kColGA = 160, kTmemCols = 256;
constexpr int kGaB = 80;  // bias-gradient column of GA
// Clock cycles a CTA waits for its products before it reports
// FV_ERR_TIMEOUT (about one second at 2 GHz).
constexpr long long kMlpWait = 2000000000ll;
constexpr uint16_t kBf16One = 0x3F80;

__host__ __device__ constexpr int kmajor(int row, int col, int K) {
  return (row >> 3) * (K * 16) + (col >> 3) * 128 + (row & 7) * 16 + (col & 7) * 2;
}

// Instruction descriptor of kind::f16 with FP32 accumulators and BF16
// operands; a_mn / b_mn select MN-major (transposed) A / B (bits 15, 16).
__host__ __device__ constexpr uint32_t idesc(int M, int N, int a_mn, int b_mn) {
  return tc_idesc_bf16(M, N) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16);
}

struct MlpArgs {
  const float* params;
  const float* x;       // rows x 16
  const float* t;       // rows x 4 (training)
  int64_t rows;
  float dy_scale;       // 2 / (4 B)
  float* y;             // rows x 4 (forward only)
  float* part;          // [grid][kMlpParams] partial gradients (training)
  float* part_loss;     // [grid] partial sums of squared residuals (training)
  unsigned int* status;
};

// 8 floats -> 8 BF16 (16 bytes) into a shared-memory operand.
__device__ __forceinline__ void st_bf16x8(unsigned char* dst, const float* v) {
  uint4 u;
  u.x = pack_bf16(v[0], v[1]);
  u.y = pack_bf16(v[2], v[3]);
  u.z = pack_bf16(v[4], v[5]);
  u.w = pack_bf16(v[6], v[7]);
  *reinterpret_cast<uint4*>(dst) = u;
}

// Offset of the 16-byte chunk of features [8c, 8c+8) of sample row t in a
// paired buffer region starting `at` bytes into the group.
__device__ __forceinline__ int prow(int t, int at, int c) {
  return (t >> 3) * kGroup + at + c * 128 + (t & 7) * 16;
}

template <bool TRAIN>
__global__ void __launch_bounds__(kRows, 2) mlp_kernel(MlpArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ alignas(8) uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ float red[kRows];
  const int tid = threadIdx.x, warp = tid >> 5;
  float* bias = reinterpret_cast<float*>(sm + kBias);

  // weights as BF16 K-major tiles; biases
  for (int i = tid; i < 64 * 16; i += kRows)
    *reinterpret_cast<uint16_t*>(sm + kW1 + kmajor(i >> 4, i & 15, 16)) =
        f32_to_bf16(a.params[kOffW1 + i]);
  for (int i = tid; i < 64 * 64; i += kRows)
    *reinterpret_cast<uint16_t*>(sm + kW2 + kmajor(i >> 6, i & 63, 64)) =
        f32_to_bf16(a.params[kOffW2 + i]);
  for (int i = tid; i < 16 * 64; i += kRows)
    *reinterpret_cast<uint16_t*>(sm + kW3 + kmajor(i >> 6, i & 63, 64)) =
        i < 4 * 64 ? f32_to_bf16(a.params[kOffW3 + i]) : (uint16_t)0;
  for (int i = tid; i < 132; i += kRows)
    bias[i] = i < 64 ? a.params[kOffB1 + i]
                     : (i < 128 ? a.params[kOffB2 + i - 64] : a.params[kOffB3 + i - 128]);
  if (TRAIN) {
    // the constant rows: ones at feature 80 of PC (B of GA) and at row 64 of
    // PB (A of GW3), zeros around them
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < 16 * 16; i += kRows) {  // 16 groups x 16 chunks of 16 B
      const int g = i >> 4, c = i & 15;
      *reinterpret_cast<uint4*>(sm + kPC + g * kGroup + kOnesC + c * 16) = z;
    }
    for (int i = tid; i < 16 * 64; i += kRows) {
      const int g = i >> 6, c = i & 63;
      *reinterpret_cast<uint4*>(sm + kPB + g * kGroup + kOnesB + c * 16) = z;
    }
    __syncthreads();
    if (tid < 16 * 8) {
      const int g = tid >> 3, r = tid & 7;
      *reinterpret_cast<uint16_t*>(sm + kPC + g * kGroup + kOnesC + r * 16) = kBf16One;
      *reinterpret_cast<uint16_t*>(sm + kPB + g * kGroup + kOnesB + r * 16) = kBf16One;
    }
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tc_alloc(&tslot, kTmemCols);
  fence_proxy_async_smem();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tm = tslot;
  const uint32_t lane_base = tm + ((uint32_t)(warp * 32) << 16);  // this warp's lanes
  const uint32_t tW = lane_base + kColW, tZ2 = lane_base + kColZ2;
  const uint32_t tG3 = lane_base + kColG3, tGA = lane_base + kColGA;

  uint32_t parity = 0u;
  bool failed = false;
  int outstanding = 0;  // a commit not yet waited for (only after a failure)
  // operands written by every thread -> visible to the tensor cores; TMEM
  // reads done; the failure flag made uniform
  auto handoff = [&]() {
    fence_proxy_async_smem();
    tc_fence_before_sync();
    failed = __syncthreads_or(failed);
    tc_fence_after_sync();
  };
  auto commit_wait = [&]() {
    if (failed) return;
    if (tid == 0) tc_commit(&bar);
    if (!mbar_wait_sleep(&bar, parity, kMlpWait)) {
      failed = true;
      outstanding = 1;
    } else {
      parity ^= 1u;
    }
    // uniform in the warp before its collective TMEM loads
    failed = __any_sync(0xffffffffu, failed);
    tc_fence_after_sync();
  };
  auto issue_z1 = [&](uint32_t dcol) {  // Z1 = X W1^T (K = 16)
    tc_mma_bf16(tm + dcol, tc_smem_desc(sm + kPC + kXoff, 128, kGroup),
                tc_smem_desc(sm + kW1, 128, 256), idesc(kRows, 64, 0, 0), 0);
  };

  const int64_t ntiles = (a.rows + kRows - 1) / kRows;
  float4 xv[4], tv = make_float4(0.f, 0.f, 0.f, 0.f);
  auto load_rows = [&](int64_t tile) {
    const int64_t r = tile * kRows + tid;
    const bool ok = tile < ntiles && r < a.rows;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      xv[i] = ok ? __ldg(reinterpret_cast<const float4*>(a.x + r * 16) + i)
                 : make_float4(0.f, 0.f, 0.f, 0.f);
    if (TRAIN) tv = ok ? __ldg(reinterpret_cast<const float4*>(a.t + r * 4))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  load_rows(blockIdx.x);
  float loss = 0.f;
  bool first = true;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row = tile * kRows + tid;
    const bool valid = row < a.rows;
    const float4 tcur = tv;
    {  // X -> PC
      float v[16] = {xv[0].x, xv[0].y, xv[0].z, xv[0].w, xv[1].x, xv[1].y, xv[1].z, xv[1].w,
                     xv[2].x, xv[2].y, xv[2].z, xv[2].w, xv[3].x, xv[3].y, xv[3].z, xv[3].w};
      st_bf16x8(sm + kPC + prow(tid, kXoff, 0), v);
      st_bf16x8(sm + kPC + prow(tid, kXoff, 1), v + 8);
    }
    load_rows(tile + gridDim.x);  // the next tile's rows arrive during this one
    handoff();
    if (tid == 0 && !failed) issue_z1(kColW);
    commit_wait();
    // ---- H1 = gelu(Z1 + b1) -> PC
    if (!failed) {
#pragma unroll
      for (int c = 0; c < 64; c += 16) {
        float v[16];
        tc_ld16(tW + c, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = gelu_f(v[i] + bias[c + i]);
        st_bf16x8(sm + kPC + prow(tid, 0, c >> 3), v);
        st_bf16x8(sm + kPC + prow(tid, 0, (c >> 3) + 1), v + 8);
      }
    }
    handoff();
    if (tid == 0 && !failed) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)  // Z2 = H1 W2^T (K = 64)
        tc_mma_bf16(tm + kColZ2, tc_smem_desc(sm + kPC + kk * 256, 128, kGroup),
                    tc_smem_desc(sm + kW2 + kk * 256, 128, 1024), idesc(kRows, 64, 0, 0), kk > 0);
    }
    commit_wait();
    // ---- H2 = gelu(Z2 + b2) -> PB
    if (!failed) {
#pragma unroll
      for (int c = 0; c < 64; c += 16) {
        float v[16];
        tc_ld16(tZ2 + c, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = gelu_f(v[i] + bias[64 + c + i]);
        st_bf16x8(sm + kPB + prow(tid, 0, c >> 3), v);
        st_bf16x8(sm + kPB + prow(tid, 0, (c >> 3) + 1), v + 8);
      }
    }
    handoff();
    if (tid == 0 && !failed) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)  // Y = H2 W3^T (N = 16, rows 4..15 of W3 zero)
        tc_mma_bf16(tm + kColW, tc_smem_desc(sm + kPB + kk * 256, 128, kGroup),
                    tc_smem_desc(sm + kW3 + kk * 256, 128, 1024), idesc(kRows, 16, 0, 0), kk > 0);
    }
    commit_wait();
    // ---- Y, residual, dY
    float yv[4] = {0.f, 0.f, 0.f, 0.f};
    if (!failed) tc_ld4(tW, yv);
#pragma unroll
    for (int o = 0; o < 4; ++o) yv[o] += bias[128 + o];
    if (!TRAIN) {
      if (valid && !failed)
        *reinterpret_cast<float4*>(a.y + row * 4) = make_float4(yv[0], yv[1], yv[2], yv[3]);
      handoff();  // this tile's TMEM reads done before the next tile's products
      continue;
    }
    {
      const float tt[4] = {tcur.x, tcur.y, tcur.z, tcur.w};
      float dy[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const float r = valid ? yv[o] - tt[o] : 0.f;
        loss = fmaf(r, r, loss);
        dy[o] = a.dy_scale * r;
      }
      const float zero8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      st_bf16x8(sm + kPC + prow(tid, kDYoff, 0), dy);
      st_bf16x8(sm + kPC + prow(tid, kDYoff, 1), zero8);
    }
    handoff();
    if (tid == 0 && !failed) {
      // dH2 = dY W3: B = W3 read MN-major (element (h, o) of W3^T)
      tc_mma_bf16(tm + kColW, tc_smem_desc(sm + kPC + kDYoff, 128, kGroup),
                  tc_smem_desc(sm + kW3, 1024, 128), idesc(kRows, 64, 0, 1), 0);
      // GW3 += [H2 ; 1]^T dY over the tile's samples (K = 128)
#pragma unroll
      for (int kk = 0; kk < 8; ++kk)
        tc_mma_bf16(tm + kColG3, tc_smem_desc(sm + kPB + kk * 2 * kGroup, kGroup, 128),
                    tc_smem_desc(sm + kPC + kDYoff + kk * 2 * kGroup, kGroup, 128),
                    idesc(kRows, 16, 1, 1), (first && kk == 0) ? 0 : 1);
    }
    commit_wait();
    // ---- dZ2 = dH2 . gelu'(Z2 + b2) -> PA (first half)
    if (!failed) {
#pragma unroll
      for (int c = 0; c < 64; c += 16) {
        float g[16], z[16];
        tc_ld16(tW + c, g);
        tc_ld16(tZ2 + c, z);
#pragma unroll
        for (int i = 0; i < 16; ++i) g[i] *= gelu_prime_f(z[i] + bias[64 + c + i]);
        st_bf16x8(sm + kPA + prow(tid, 0, c >> 3), g);
        st_bf16x8(sm + kPA + prow(tid, 0, (c >> 3) + 1), g + 8);
      }
    }
    handoff();
    if (tid == 0 && !failed) {
      // dH1 = dZ2 W2: B = W2 read MN-major (element (h1, h2) of W2^T)
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        tc_mma_bf16(tm + kColZ2, tc_smem_desc(sm + kPA + kk * 256, 128, kGroup),
                    tc_smem_desc(sm + kW2 + kk * 2048, 1024, 128), idesc(kRows, 64, 0, 1), kk > 0);
      issue_z1(kColW);  // Z1 once more, for gelu'(Z1)
    }
    commit_wait();
    // ---- dZ1 = dH1 . gelu'(Z1 + b1) -> PA (second half)
    if (!failed) {
#pragma unroll
      for (int c = 0; c < 64; c += 16) {
        float g[16], z[16];
        tc_ld16(tZ2 + c, g);
        tc_ld16(tW + c, z);
#pragma unroll
        for (int i = 0; i < 16; ++i) g[i] *= gelu_prime_f(z[i] + bias[c + i]);
        st_bf16x8(sm + kPA + prow(tid, 1024, c >> 3), g);
        st_bf16x8(sm + kPA + prow(tid, 1024, (c >> 3) + 1), g + 8);
      }
    }
    handoff();
    if (tid == 0 && !failed) {
      // GA += [dZ2 ; dZ1]^T [H1 ; X ; 1] over the tile's samples (K = 128)
#pragma unroll
      for (int kk = 0; kk < 8; ++kk)
        tc_mma_bf16(tm + kColGA, tc_smem_desc(sm + kPA + kk * 2 * kGroup, kGroup, 128),
                    tc_smem_desc(sm + kPC + kk * 2 * kGroup, kGroup, 128),
                    idesc(kRows, 96, 1, 1), (first && kk == 0) ? 0 : 1);
    }
    commit_wait();  // PA and PC are rewritten by the next tile
    first = false;
  }

  if (TRAIN) {
    // this CTA's partial gradient and loss
    float* pg = a.part + (int64_t)blockIdx.x * kMlpParams;
    if (!failed && !first) {
      float g3[4];
      tc_ld4(tG3, g3);
      float gb[4];
      tc_ld4(tGA + kGaB, gb);
      if (warp < 2) {  // rows 0..63: dW2, db2, dW3
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
          float v[16];
          tc_ld16(tGA + c, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) pg[kOffW2 + tid * 64 + c + i] = v[i];
        }
        pg[kOffB2 + tid] = gb[0];
#pragma unroll
        for (int o = 0; o < 4; ++o) pg[kOffW3 + o * 64 + tid] = g3[o];
      } else {  // rows 64..127: dW1, db1; row 64: db3
        float v[16];
        tc_ld16(tGA + 64, v);
        const int h = tid - 64;
#pragma unroll
        for (int i = 0; i < 16; ++i) pg[kOffW1 + h * 16 + i] = v[i];
        pg[kOffB1 + h] = gb[0];
        if (tid == 64) {
#pragma unroll
          for (int o = 0; o < 4; ++o) pg[kOffB3 + o] = g3[o];
        }
      }
    }
    red[tid] = loss;
    __syncthreads();
    if (tid == 0) {
      float s = 0.f;
      for (int i = 0; i < kRows; ++i) s += red[i];
      a.part_loss[blockIdx.x] = s;
    }
  }
  if (failed) {
    if (tid == 0) atomicOr(a.status, ST_TIMEOUT);
    // the products of a commit that was given up on get a second bounded wait
    // before their tensor memory is released
    if (outstanding) mbar_wait_bounded(&bar, parity, kMlpWait);
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  if (warp == 0) tc_dealloc(tm, kTmemCols);
}

// Sum of the CTAs' partial gradients (a fixed order: warp w takes the
// partials w, w + 8, ...; then the eight warp sums in order), then either
// the gradient out or one Adam step (Kingma & Ba 2015: m = b1 m + (1-b1) g,
// v = b2 v + (1-b2) g^2, theta -= lr mhat / (sqrt(vhat) + eps)).  Block 0
// also sums the partial losses.
struct UpdateArgs {
  const float* part;
  const float* part_loss;
  int nparts;
  float inv_n;      // 1 / (4 B)
  float* grad_out;  // gradient mode, else null
  float* params;
  float* m;
  float* v;
  float lr, b1, b2, eps, c1, c2;
  float* loss_out;
};

__global__ void __launch_bounds__(256) mlp_update_kernel(UpdateArgs u) {
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (i < kMlpParams) {
    int c = w;
    for (; c + 24 < u.nparts; c += 32) {  // four loads in flight, summed in order
      const float v0 = u.part[(int64_t)c * kMlpParams + i];
      const float v1 = u.part[(int64_t)(c + 8) * kMlpParams + i];
      const float v2 = u.part[(int64_t)(c + 16) * kMlpParams + i];
      const float v3 = u.part[(int64_t)(c + 24) * kMlpParams + i];
      s += v0;
      s += v1;
      s += v2;
      s += v3;
    }
    for (; c < u.nparts; c += 8) s += u.part[(int64_t)c * kMlpParams + i];
  }
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && i < kMlpParams) {
    float g = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) g += red[k][lane];
    if (u.grad_out) {
      u.grad_out[i] = g;
    } else {
      const float mi = u.b1 * u.m[i] + (1.f - u.b1) * g;
      const float vi = u.b2 * u.v[i] + (1.f - u.b2) * g * g;
      u.m[i] = mi;
      u.v[i] = vi;
      u.params[i] -= u.lr * (mi / u.c1) / (sqrtf(vi / u.c2) + u.eps);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 32 && u.loss_out) {
    float l = 0.f;
    for (int c = 0; c < u.nparts; ++c) l += u.part_loss[c];
    *u.loss_out = l * u.inv_n;
  }
}

}  // namespace
}  // namespace fv

// ---------------------------------------------------------------------------
// Trainer: the partial-gradient workspace and the Adam moments.
// ---------------------------------------------------------------------------
struct fv_mlp_trainer {
  cudaStream_t stream = nullptr;
  int64_t max_batch = 0;
  int grid_max = 0;   // CTAs of the network kernel (two per SM)
  void* ws = nullptr;
  float *part = nullptr, *part_loss = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  unsigned int* status = nullptr;
};

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int mlp_grid(const fv_mlp_trainer* t, int64_t batch) {
  const int64_t tiles = (batch + fv::kRows - 1) / fv::kRows;
  return (int)(tiles < t->grid_max ? tiles : t->grid_max);
}

cudaError_t launch_net(const fv_mlp_trainer* t, bool train, const float* params, const float* x,
                       const float* target, int64_t batch, float* y, int* grid_out) {
  fv::MlpArgs a;
  a.params = params;
  a.x = x;
  a.t = target;
  a.rows = batch;
  a.dy_scale = 2.0f / (4.0f * (float)batch);
  a.y = y;
  a.part = t->part;
  a.part_loss = t->part_loss;
  a.status = t->status;
  const int grid = mlp_grid(t, batch);
  if (grid_out) *grid_out = grid;
  if (train)
    fv::mlp_kernel<true><<<grid, fv::kRows, fv::kSmemBytes, t->stream>>>(a);
  else
    fv::mlp_kernel<false><<<grid, fv::kRows, fv::kSmemBytes, t->stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_update(const fv_mlp_trainer* t, int nparts, int64_t batch, float* grad_out,
                          float* params, float lr, int step, float* loss) {
  fv::UpdateArgs u;
  u.part = t->part;
  u.part_loss = t->part_loss;
  u.nparts = nparts;
  u.inv_n = 1.0f / (4.0f * (float)batch);
  u.grad_out = grad_out;
  u.params = params;
  u.m = t->m;
  u.v = t->v;
  u.lr = lr;
  u.b1 = 0.9f;
  u.b2 = 0.999f;
  u.eps = 1e-8f;
  u.c1 = grad_out ? 1.f : 1.f - powf(u.b1, (float)step);
  u.c2 = grad_out ? 1.f : 1.f - powf(u.b2, (float)step);
  u.loss_out = loss;
  fv::mlp_update_kernel<<<(fv::kMlpParams + 31) / 32, 256, 0, t->stream>>>(u);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

fv_status fv_mlp_trainer_create(fv_mlp_trainer** out, int64_t max_batch, void* stream) {
  if (!out || max_batch < 1 || max_batch > (1ll << 28)) return FV_ERR_INVALID_ARG;
  *out = nullptr;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FV_ERR_CUDA;
  // shared memory of the network kernel: two CTAs per SM
  if (cudaFuncSetAttribute(fv::mlp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           fv::kSmemBytes) != cudaSuccess ||
      cudaFuncSetAttribute(fv::mlp_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           fv::kSmemBytes) != cudaSuccess)
    return FV_ERR_CUDA;
  fv_mlp_trainer* t = new (std::nothrow) fv_mlp_trainer();
  if (!t) return FV_ERR_CUDA;
  t->stream = static_cast<cudaStream_t>(stream);
  t->max_batch = max_batch;
  t->grid_max = 2 * sms;
  const int64_t P = fv::kMlpParams;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align256(bytes);
    return o;
  };
  const size_t o_part = take(4 * (size_t)t->grid_max * P), o_pl = take(4 * (size_t)t->grid_max),
               o_grad = take(4 * P), o_m = take(4 * P), o_v = take(4 * P), o_st = take(4);
  cudaError_t e = cudaMalloc(&t->ws, off);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->ws, 0, off, t->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
  if (e != cudaSuccess) {
    if (t->ws) cudaFree(t->ws);
    delete t;
    return FV_ERR_CUDA;
  }
  char* w = static_cast<char*>(t->ws);
  t->part = (float*)(w + o_part);
  t->part_loss = (float*)(w + o_pl);
  t->grad = (float*)(w + o_grad);
  t->m = (float*)(w + o_m);
  t->v = (float*)(w + o_v);
  t->status = (unsigned int*)(w + o_st);
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

fv_status fv_mlp_trainer_status(fv_mlp_trainer* t) {
  if (!t) return FV_ERR_INVALID_ARG;
  unsigned int bits = 0;
  cudaError_t e = cudaStreamSynchronize(t->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&bits, t->status, sizeof(bits), cudaMemcpyDeviceToHost, t->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->status, 0, sizeof(bits), t->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(t->stream);
  if (e != cudaSuccess) return FV_ERR_CUDA;
  return (bits & fv::ST_TIMEOUT) ? FV_ERR_TIMEOUT : FV_OK;
}

fv_status fv_mlp_forward(fv_mlp_trainer* t, const float* params, const float* x, int64_t batch,
                         float* y) {
  if (!t || !params || !x || !y || batch < 1 || batch > t->max_batch) return FV_ERR_INVALID_ARG;
  if (((uintptr_t)x | (uintptr_t)y) & 15u) return FV_ERR_ALIGNMENT;
  cudaError_t e = launch_net(t, false, params, x, nullptr, batch, y, nullptr);
  return e == cudaSuccess ? FV_OK : FV_ERR_CUDA;
}

fv_status fv_mlp_grad(fv_mlp_trainer* t, const float* params, const float* x,
                      const float* target, int64_t batch, float* grad, float* loss) {
  if (!t || !params || !x || !target || !grad || !loss || batch < 1 || batch > t->max_batch)
    return FV_ERR_INVALID_ARG;
  if (((uintptr_t)x | (uintptr_t)target) & 15u) return FV_ERR_ALIGNMENT;
  int grid = 0;
  cudaError_t e = launch_net(t, true, params, x, target, batch, nullptr, &grid);
  if (e == cudaSuccess) e = launch_update(t, grid, batch, grad, nullptr, 0.f, 1, loss);
  return e == cudaSuccess ? FV_OK : FV_ERR_CUDA;
}

fv_status fv_mlp_train_step(fv_mlp_trainer* t, float* params, const float* x, const float* target,
                            int64_t batch, float lr, int step, float* loss) {
  return fv_mlp_train_steps(t, params, x, target, batch, batch, step, 1, lr, loss);
}

fv_status fv_mlp_train_steps(fv_mlp_trainer* t, float* params, const float* x,
                             const float* target, int64_t n_samples, int64_t batch,
                             int first_step, int n_steps, float lr, float* losses) {
  if (!t || !params || !x || !target || batch < 1 || batch > t->max_batch ||
      n_samples < batch || first_step < 1 || n_steps < 0 || !(lr > 0.f))
    return FV_ERR_INVALID_ARG;
  if (((uintptr_t)x | (uintptr_t)target) & 15u) return FV_ERR_ALIGNMENT;
  const int64_t nb = n_samples / batch;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
    const int step = first_step + k;
    const int64_t r0 = ((int64_t)(step - 1) % nb) * batch;
    int grid = 0;
    e = launch_net(t, true, params, x + r0 * 16, target + r0 * 4, batch, nullptr, &grid);
    if (e == cudaSuccess)
      e = launch_update(t, grid, batch, nullptr, params, lr, step, losses ? losses + k : nullptr);
  }
  return e == cudaSuccess ? FV_OK : FV_ERR_CUDA;
}

}  // extern "C"
