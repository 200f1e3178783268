// nrc.cu - neural radiance cache: frequency encoding, fused tcgen05 MLP
// inference and training (forward, backward, weight gradients accumulated in
// tensor memory), Adam on FP32 master weights.
//
// Network: 96 inputs (81 used) -> 64 -> 64 -> 64 -> 64 -> 3, ReLU hidden
// layers, exp output; BF16 weights and activations, FP32 accumulation.
// Loss: mean over samples and channels of (y - t)^2 / (sg(y)^2 + 0.01).
// The paper has no learned component; this cache terminates paths after a
// fixed bounce and is trained online on radiance the tracer itself produces.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "nrc_internal.cuh"
#include "rtb_internal.cuh"
#include "tc.cuh"

namespace rtb {

// ---------------------------------------------------------------------------
// parameter layouts
// ---------------------------------------------------------------------------
// FP32 master parameters (oracle layout): W0[64][96] W1[64][64] W2 W3 W4[3][64],
// then b0[64] b1 b2 b3 b4[3].
__host__ __device__ constexpr int off_w(int l) { return l == 0 ? 0 : 6144 + 4096 * (l - 1); }
__host__ __device__ constexpr int off_b(int l) { return kNW + 64 * l; }
__host__ __device__ constexpr int d_in(int l) { return l == 0 ? 96 : 64; }
__host__ __device__ constexpr int d_out(int l) { return l == 4 ? 3 : 64; }

// Packed BF16 copies (row-major) read by the kernels, then FP32 biases.
// forward W_l as [out][in] (W4 padded to 16 rows), backward W_l^T as
// [in][out] (W4^T padded to 16 columns).
constexpr int kPW0 = 0, kPW1 = 6144, kPW2 = 10240, kPW3 = 14336, kPW4 = 18432;   // W4: 16 x 64
constexpr int kPT1 = 19456, kPT2 = 23552, kPT3 = 27648, kPT4 = 31744;             // T4: 64 x 16
constexpr int kPackedBf16 = 32768;                                                 // 64 KB
constexpr int kPackedBias = 4 * 64 + 16;
constexpr size_t kPackedBytes = kPackedBf16 * 2 + kPackedBias * 4;

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_float(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// ---------------------------------------------------------------------------
// encoding: 3 normalised position values, normal (3), view direction (3),
// sin and cos of 2^k pi x_hat_j for k = 0..11 -> 81 values, zero-padded to 96
// ---------------------------------------------------------------------------
__device__ __forceinline__ void encode81(const float* pnv, const float* lo, const float* inv_ext, float* f) {
  float xh[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    xh[j] = (pnv[j] - lo[j]) * inv_ext[j];
    f[j] = xh[j];
    f[3 + j] = pnv[3 + j];
    f[6 + j] = pnv[6 + j];
  }
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    float sc = (float)(1 << k);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float s, c;
      sincospif(sc * xh[j], &s, &c);
      f[9 + 6 * k + j] = s;
      f[9 + 6 * k + 3 + j] = c;
    }
  }
#pragma unroll
  for (int k = 81; k < 96; ++k) f[k] = 0.f;
}

// Writes 8 consecutive features (columns 8c..8c+7) of row r as one 16-byte
// chunk of a K-major canonical tile.
__device__ __forceinline__ void store_chunk(uint8_t* tile, int r, int c, int K, const float* v8) {
  uint4 q;
  q.x = (uint32_t)bf16_bits(v8[0]) | ((uint32_t)bf16_bits(v8[1]) << 16);
  q.y = (uint32_t)bf16_bits(v8[2]) | ((uint32_t)bf16_bits(v8[3]) << 16);
  q.z = (uint32_t)bf16_bits(v8[4]) | ((uint32_t)bf16_bits(v8[5]) << 16);
  q.w = (uint32_t)bf16_bits(v8[6]) | ((uint32_t)bf16_bits(v8[7]) << 16);
  *(uint4*)(tile + tc::core_off(r, 8 * c, K)) = q;
}

// Copies a row-major [R][K] bf16 matrix from global memory into a K-major
// canonical tile (16-byte chunks).
__device__ __forceinline__ void load_tile(uint8_t* tile, const uint16_t* __restrict__ g, int R, int K) {
  int chunks = R * (K / 8);
  for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
    int r = i / (K / 8), c = i % (K / 8);
    uint4 q = *(const uint4*)(g + (size_t)r * K + 8 * c);
    *(uint4*)(tile + tc::core_off(r, 8 * c, K)) = q;
  }
}

// ---------------------------------------------------------------------------
// inference: records (p, n, v, weight, pixel) -> pixel += weight * exp(MLP)
// 128 threads, one sample per thread, one 128-sample tile at a time.
// ---------------------------------------------------------------------------
constexpr int kInferThreads = 128;
constexpr int kInferTmemCols = 64;
// dynamic shared memory (bytes), 1 KB aligned sections
constexpr int kSmW0 = 0, kSmW1 = 12288, kSmW2 = 20480, kSmW3 = 28672, kSmW4 = 36864;   // 2 KB
constexpr int kSmBias = 38912;                                                         // 272 floats
constexpr int kSmA = 40960;                                                            // 24 KB
constexpr int kSmMisc = 65536;                                                         // mbarrier, tmem slot, flags
constexpr int kInferSmem = kSmMisc + 64;

__device__ __forceinline__ void fb_add(float* fb, float* target, int pixel, float r, float g, float b) {
  float* p = pixel >= 0 ? fb + 3 * (size_t)pixel : target + 3 * (size_t)(~pixel);
  atomicAdd(p, r);
  atomicAdd(p + 1, g);
  atomicAdd(p + 2, b);
}

__global__ void __launch_bounds__(kInferThreads) k_nrc_infer(NrcDevice nd, const float4* __restrict__ recs,
                                                            const unsigned* __restrict__ count, unsigned cap,
                                                            float* __restrict__ fb, float* __restrict__ out3,
                                                            unsigned* status, float* const* __restrict__ fbs) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* mbar = (uint64_t*)(sm + kSmMisc);
  uint32_t* tslot = (uint32_t*)(sm + kSmMisc + 8);
  int* abort_flag = (int*)(sm + kSmMisc + 16);
  float* bias = (float*)(sm + kSmBias);
  int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tc::alloc(tc::smem_u32(tslot), kInferTmemCols);
  const uint16_t* pw = (const uint16_t*)nd.packed;
  load_tile(sm + kSmW0, pw + kPW0, 64, 96);
  load_tile(sm + kSmW1, pw + kPW1, 64, 64);
  load_tile(sm + kSmW2, pw + kPW2, 64, 64);
  load_tile(sm + kSmW3, pw + kPW3, 64, 64);
  load_tile(sm + kSmW4, pw + kPW4, 16, 64);
  const float* gb = (const float*)(pw + kPackedBf16);
  for (int i = tid; i < kPackedBias; i += blockDim.x) bias[i] = gb[i];
  if (tid == 0) {
    tc::mbar_init(tc::smem_u32(mbar), 1);
    *abort_flag = 0;
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  uint32_t tmem = *tslot;
  uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t mb = tc::smem_u32(mbar);
  uint32_t sA = tc::smem_u32(sm + kSmA);
  const uint32_t sW[5] = {tc::smem_u32(sm + kSmW0), tc::smem_u32(sm + kSmW1), tc::smem_u32(sm + kSmW2),
                          tc::smem_u32(sm + kSmW3), tc::smem_u32(sm + kSmW4)};
  unsigned n = min(*count, cap);
  unsigned tiles = (n + 127) / 128;
  uint32_t phase = 0;
  float lo[3] = {nd.lo[0], nd.lo[1], nd.lo[2]}, ie[3] = {nd.inv_ext[0], nd.inv_ext[1], nd.inv_ext[2]};
  for (unsigned tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    unsigned row = tile * 128 + tid;
    bool valid = row < n;
    float f[96];
    float wr = 0.f, wg = 0.f, wb = 0.f;
    int pixel = 0, frame = 0;
    if (valid) {
      float4 q0 = recs[4 * (size_t)row], q1 = recs[4 * (size_t)row + 1], q2 = recs[4 * (size_t)row + 2],
             q3 = recs[4 * (size_t)row + 3];
      float pnv[9] = {q0.x, q0.y, q0.z, q1.x, q1.y, q1.z, q2.x, q2.y, q2.z};
      encode81(pnv, lo, ie, f);
      pixel = __float_as_int(q0.w);
      frame = __float_as_int(q3.w);
      wr = q3.x;
      wg = q3.y;
      wb = q3.z;
    } else {
#pragma unroll
      for (int k = 0; k < 96; ++k) f[k] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < 12; ++c) store_chunk(sm + kSmA, tid, c, 96, f + 8 * c);
    tc::fence_proxy_async();
    __syncthreads();
    for (int l = 0; l < 5; ++l) {
      int N = l < 4 ? 64 : 16;
      if (tid == 0) {
        tc::fence_after_sync();
        tc::gemm(tmem, sA, sW[l], d_in(l), tc::idesc_bf16_f32(128, N), false);
        tc::commit(mb);
      }
      bool ok = tc::mbar_wait(mb, phase);
      phase ^= 1;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(status, kErrNrcTimeout);
        goto done;
      }
      tc::fence_after_sync();
      if (l < 4) {
        float h[64];
#pragma unroll
        for (int c = 0; c < 4; ++c) tc::ld16(lane_addr + 16 * c, h + 16 * c);
#pragma unroll
        for (int k = 0; k < 64; ++k) h[k] = fmaxf(h[k] + bias[64 * l + k], 0.f);
#pragma unroll
        for (int c = 0; c < 8; ++c) store_chunk(sm + kSmA, tid, c, 64, h + 8 * c);
        tc::fence_before_sync();
        tc::fence_proxy_async();
        __syncthreads();
      } else {
        float o[16];
        tc::ld16(lane_addr, o);
        float y0 = expf(o[0] + bias[256]), y1 = expf(o[1] + bias[257]), y2 = expf(o[2] + bias[258]);
        if (valid) {
          if (out3) {
            out3[3 * (size_t)row] = y0;
            out3[3 * (size_t)row + 1] = y1;
            out3[3 * (size_t)row + 2] = y2;
          }
          if (fbs) fb_add(fbs[frame], nd.target, pixel, wr * y0, wg * y1, wb * y2);
          else if (fb) fb_add(fb, nd.target, pixel, wr * y0, wg * y1, wb * y2);
        }
        tc::fence_before_sync();
        __syncthreads();
      }
    }
  }
done:
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::dealloc(tmem, kInferTmemCols);
}

// ---------------------------------------------------------------------------
// training: forward (activations kept), loss gradient, backward; weight and
// bias gradients accumulate in tensor memory over the CTA's tiles, then go
// to its own row of the gradient buffer.  One CTA per SM (its 512
// tensor-memory columns), 128 samples a tile, one sample a thread.
//
// Every activation is stored once, row by row (a sample's features in
// 16-byte chunks, the K-major layout of the forward MMAs).  The
// weight-gradient MMAs, whose K is the batch, read the same tiles as
// MN-major operands, so no transposed copy is made.  The activation tiles
// carry a constant column of ones past their features, so each weight-
// gradient MMA also sums the backward signal over the batch: the bias
// gradient of that layer.
// ---------------------------------------------------------------------------
constexpr int kTrainThreads = 128;
constexpr int kTrainTmemCols = 512;
// activation tiles: width (features + the ones column, padded to 8)
constexpr int kXW = 104;    // X: 96 features, ones at column 96
constexpr int kHW = 80;     // H1..H4: 64 features, ones at column 64
// tensor-memory columns (16-aligned)
constexpr int kTcAcc = 0;      // 64: forward / backward accumulator (M = 128)
constexpr int kTcDW0 = 64;     // 104: dW0 | dB0 (M = 64, N = 104)
constexpr int kTcDW1 = 176;    // 80 each at 176, 256, 336: dW_l | dB_l (M = 64, N = 80)
constexpr int kTcDW4 = 416;    // 16: dW4^T (M = 64, N = 16)
// shared memory (bytes)
constexpr int kTsW0 = 0, kTsW1 = 12288, kTsW2 = 20480, kTsW3 = 28672, kTsW4 = 36864;   // forward, 38 KB
constexpr int kTsT1 = 38912, kTsT2 = 47104, kTsT3 = 55296, kTsT4 = 63488;              // backward, 26 KB
constexpr int kTsX = 65536;                        // X [128][104]: 26 KB
constexpr int kTsH = kTsX + 128 * kXW * 2;         // H1..H4 [128][80]: 4 x 20 KB
constexpr int kTsDZ = kTsH + 4 * 128 * kHW * 2;    // dZ [128][64] (dZ5: [128][16]): 16 KB
constexpr int kTsBias = kTsDZ + 16384;             // 272 floats
constexpr int kTsDB = kTsBias + 1088;              // dB4 of each warp: 4 x 4 floats
constexpr int kTsMisc = kTsDB + 64;                // mbarrier, tmem slot, loss of each warp
// the allocation ends 32 KB past the last tile, so that no operand
// descriptor can reach past it whatever its strides
constexpr int kTrainSmem = kTsMisc + 64 + 32768;
static_assert(kTrainSmem <= 227 * 1024, "the training CTA's shared memory exceeds the per-block limit");

// One CTA's gradient row: the kNP parameter gradients (oracle layout), then
// the loss, padded to whole float4.
constexpr int kGPRow = (kNP + 1 + 3) / 4 * 4;

__device__ __forceinline__ void store16(float* dst, const float* v) {   // dst 16-byte aligned
  float4* d = (float4*)dst;
  d[0] = make_float4(v[0], v[1], v[2], v[3]);
  d[1] = make_float4(v[4], v[5], v[6], v[7]);
  d[2] = make_float4(v[8], v[9], v[10], v[11]);
  d[3] = make_float4(v[12], v[13], v[14], v[15]);
}

// Lane of row m of an M = 64 accumulator: 16 rows in each 32-lane quarter.
__device__ __forceinline__ int m64_row_of_lane(int lane) { return (lane & 31) < 16 ? (lane >> 5) * 16 + (lane & 31) : -1; }

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The constant columns of a [128][width] activation tile: ones at column
// `col`, zeros up to the width (chunks from col / 8 on).
__device__ __forceinline__ void fill_ones(uint8_t* tile, int width, int col) {
  for (int i = threadIdx.x; i < 128 * (width - col) / 8; i += blockDim.x) {
    const int r = i / ((width - col) / 8), c = col / 8 + i % ((width - col) / 8);
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (c == col / 8) v[0] = 1.f;
    store_chunk(tile, r, c, width, v);
  }
}

__global__ void __launch_bounds__(kTrainThreads, 1) k_nrc_train(NrcDevice nd, const float4* __restrict__ recs,
                                                                const float* __restrict__ targets,
                                                                const unsigned* __restrict__ count, unsigned cap,
                                                                float* __restrict__ gpart, unsigned* status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* mbar = (uint64_t*)(sm + kTsMisc);
  uint32_t* tslot = (uint32_t*)(sm + kTsMisc + 8);
  float* s_loss = (float*)(sm + kTsMisc + 16);   // [4]
  float* bias = (float*)(sm + kTsBias);
  float* db4 = (float*)(sm + kTsDB);              // [warp][4]
  int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::alloc(tc::smem_u32(tslot), kTrainTmemCols);
  const uint16_t* pw = (const uint16_t*)nd.packed;
  load_tile(sm + kTsW0, pw + kPW0, 64, 96);
  load_tile(sm + kTsW1, pw + kPW1, 64, 64);
  load_tile(sm + kTsW2, pw + kPW2, 64, 64);
  load_tile(sm + kTsW3, pw + kPW3, 64, 64);
  load_tile(sm + kTsW4, pw + kPW4, 16, 64);
  load_tile(sm + kTsT1, pw + kPT1, 64, 64);
  load_tile(sm + kTsT2, pw + kPT2, 64, 64);
  load_tile(sm + kTsT3, pw + kPT3, 64, 64);
  load_tile(sm + kTsT4, pw + kPT4, 64, 16);
  fill_ones(sm + kTsX, kXW, 96);
  for (int l = 0; l < 4; ++l) fill_ones(sm + kTsH + l * 128 * kHW * 2, kHW, 64);
  const float* gb = (const float*)(pw + kPackedBf16);
  for (int i = tid; i < kPackedBias; i += blockDim.x) bias[i] = gb[i];
  if (tid < 16) db4[tid] = 0.f;
  if (tid == 0) {
    tc::mbar_init(tc::smem_u32(mbar), 1);
    *s_loss = 0.f;
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  uint32_t tmem = *tslot;
  uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t mb = tc::smem_u32(mbar);
  const uint32_t sW[5] = {tc::smem_u32(sm + kTsW0), tc::smem_u32(sm + kTsW1), tc::smem_u32(sm + kTsW2),
                          tc::smem_u32(sm + kTsW3), tc::smem_u32(sm + kTsW4)};
  const uint32_t sT[5] = {0u, tc::smem_u32(sm + kTsT1), tc::smem_u32(sm + kTsT2), tc::smem_u32(sm + kTsT3),
                          tc::smem_u32(sm + kTsT4)};
  // the activation entering layer l: X, then H1..H4, and its tile width
  uint32_t sAct[5];
  sAct[0] = tc::smem_u32(sm + kTsX);
  for (int l = 1; l <= 4; ++l) sAct[l] = tc::smem_u32(sm + kTsH + (l - 1) * 128 * kHW * 2);
  const uint32_t sDZ = tc::smem_u32(sm + kTsDZ);
  unsigned n = min(*count, cap);
  unsigned tiles = (n + 127) / 128;
  float inv_n3 = n > 0 ? 1.0f / (3.0f * (float)n) : 0.f;
  uint32_t phase = 0;
  bool first = true;
  float loss_acc = 0.f;
  bool aborted = false;
  float lo[3] = {nd.lo[0], nd.lo[1], nd.lo[2]}, ie[3] = {nd.inv_ext[0], nd.inv_ext[1], nd.inv_ext[2]};

#define RTB_WAIT()                                   \
  {                                                  \
    bool ok_ = tc::mbar_wait(mb, phase);             \
    phase ^= 1;                                      \
    if (__syncthreads_or(!ok_)) {                    \
      if (tid == 0) atomicOr(status, kErrNrcTimeout); \
      aborted = true;                                \
      goto done;                                     \
    }                                                \
    tc::fence_after_sync();                          \
  }

  for (unsigned tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    unsigned row = tile * 128 + tid;
    bool valid = row < n;
    uint32_t mask[4][2];   // ReLU masks of the 4 hidden layers (64 bits each)
    float tr = 0.f, tg = 0.f, tb = 0.f;
    {
      float f[96];
      if (valid) {
        float4 q0 = recs[3 * (size_t)row], q1 = recs[3 * (size_t)row + 1], q2 = recs[3 * (size_t)row + 2];
        float pnv[9] = {q0.x, q0.y, q0.z, q1.x, q1.y, q1.z, q2.x, q2.y, q2.z};
        encode81(pnv, lo, ie, f);
        int slot = __float_as_int(q0.w);
        tr = targets[3 * (size_t)slot];
        tg = targets[3 * (size_t)slot + 1];
        tb = targets[3 * (size_t)slot + 2];
      } else {
#pragma unroll
        for (int k = 0; k < 96; ++k) f[k] = 0.f;
      }
#pragma unroll
      for (int c = 0; c < 12; ++c) store_chunk(sm + kTsX, tid, c, kXW, f + 8 * c);
    }
    tc::fence_proxy_async();
    __syncthreads();
    // forward: Z_{l+1} = Act_l W_l^T (A = the activation tile, K-major)
    float o[16];
    for (int l = 0; l < 5; ++l) {
      int N = l < 4 ? 64 : 16;
      if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t sbo_a = (uint32_t)((l == 0 ? kXW : kHW) / 8) * 128u;
        const uint32_t sbo_b = (uint32_t)(d_in(l) / 8) * 128u;
        tc::gemm_kk(tmem + kTcAcc, sAct[l], sbo_a, sW[l], sbo_b, d_in(l), tc::idesc_bf16_f32(128, N), false);
        tc::commit(mb);
      }
      RTB_WAIT();
      if (l < 4) {
        float h[64];
#pragma unroll
        for (int c = 0; c < 4; ++c) tc::ld16(lane_addr + kTcAcc + 16 * c, h + 16 * c);
        mask[l][0] = mask[l][1] = 0u;
#pragma unroll
        for (int k = 0; k < 64; ++k) {
          float z = h[k] + bias[64 * l + k];
          bool pos = valid && z > 0.f;
          mask[l][k >> 5] |= (pos ? 1u : 0u) << (k & 31);
          h[k] = pos ? z : 0.f;
        }
        uint8_t* hl = sm + kTsH + l * 128 * kHW * 2;
#pragma unroll
        for (int c = 0; c < 8; ++c) store_chunk(hl, tid, c, kHW, h + 8 * c);
        tc::fence_before_sync();
        tc::fence_proxy_async();
        __syncthreads();
      } else {
        tc::ld16(lane_addr + kTcAcc, o);
        tc::fence_before_sync();
      }
    }
    // loss gradient at the exp output: dL/dz5 = 2 (y - t) / (y^2 + 0.01) / (3n) * y,
    // stored in BF16; the output bias gradient sums the stored values
    {
      float g[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) g[k] = 0.f;
      if (valid) {
        float t3[3] = {tr, tg, tb};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float y = expf(o[c] + bias[256 + c]);
          float den = y * y + 0.01f;
          float dy = y - t3[c];
          loss_acc += dy * dy / den * inv_n3;
          g[c] = 2.f * dy / den * inv_n3 * y;
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float s = warp_sum(bf16_float(bf16_bits(g[c])));
        if (lane == 0) db4[4 * warp + c] += s;
      }
      store_chunk(sm + kTsDZ, tid, 0, 16, g);
      store_chunk(sm + kTsDZ, tid, 1, 16, g + 8);
      tc::fence_proxy_async();
      __syncthreads();
    }
    // backward: layer 4 -> 0.  dW_l | dB_l [M = out][N = in + ones] += dZ^T Act_l,
    // both operands MN-major over the batch; dAct_l = dZ W_l (K-major)
    for (int l = 4; l >= 0; --l) {
      if (tid == 0) {
        tc::fence_after_sync();
        if (l == 4) {
          // dW4^T [64 in][16 out] += H4^T dZ5: A = H4 (M = in), B = dZ5 (N = out)
          tc::gemm_mn(tmem + kTcDW4, sAct[4], (uint32_t)(kHW / 8) * 128u, sDZ, 2u * 128u, 128,
                      tc::idesc_bf16_f32_mn(64, 16), !first);
          // dH4 = dZ5 W4 (A: dZ5 [128][16], B: W4^T [64][16])
          tc::gemm(tmem + kTcAcc, sDZ, sT[4], 16, tc::idesc_bf16_f32(128, 64), false);
        } else {
          // dW_l | dB_l += dZ^T [Act_l | 1]: A = dZ (M = out), B = Act_l (N = in + ones)
          const uint32_t col = l == 0 ? kTcDW0 : kTcDW1 + 80 * (l - 1);
          const int width = l == 0 ? kXW : kHW;
          tc::gemm_mn(tmem + col, sDZ, 8u * 128u, sAct[l], (uint32_t)(width / 8) * 128u, 128,
                      tc::idesc_bf16_f32_mn(64, width), !first);
          if (l > 0) tc::gemm(tmem + kTcAcc, sDZ, sT[l], 64, tc::idesc_bf16_f32(128, 64), false);
        }
        tc::commit(mb);
      }
      RTB_WAIT();
      if (l == 0) break;
      // dZ_l = dH_l * relu'(z_l), stored in BF16 for both of its MMAs
      float g[64];
#pragma unroll
      for (int c = 0; c < 4; ++c) tc::ld16(lane_addr + kTcAcc + 16 * c, g + 16 * c);
#pragma unroll
      for (int k = 0; k < 64; ++k) g[k] = ((mask[l - 1][k >> 5] >> (k & 31)) & 1u) ? g[k] : 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) store_chunk(sm + kTsDZ, tid, c, 64, g + 8 * c);
      tc::fence_before_sync();
      tc::fence_proxy_async();
      __syncthreads();
    }
    tc::fence_before_sync();
    __syncthreads();
    first = false;
  }
done:
  // this CTA's gradients and loss: its own row of gpart (plain stores; the
  // Adam kernel sums the rows in a fixed order).  A CTA without a tile, or
  // one whose wait timed out, writes zeros.
  float* gp = gpart + (size_t)blockIdx.x * kGPRow;
  const bool have = !aborted && !first;
  if (have) {
    tc::fence_after_sync();
    int m = m64_row_of_lane(tid);
    float v[16];
    // dW0 | dB0 (M = 64 x N = 104): columns 0..95 the weights, 96 the bias
    for (int c = 0; c < 7; ++c) {
      tc::ld16(lane_addr + kTcDW0 + 16 * c, v);
      if (m >= 0) {
        if (c < 6) store16(gp + off_w(0) + m * 96 + 16 * c, v);
        else gp[off_b(0) + m] = v[0];
      }
    }
    for (int l = 1; l <= 3; ++l)
      for (int c = 0; c < 5; ++c) {
        tc::ld16(lane_addr + kTcDW1 + 80 * (l - 1) + 16 * c, v);
        if (m >= 0) {
          if (c < 4) store16(gp + off_w(l) + m * 64 + 16 * c, v);
          else gp[off_b(l) + m] = v[0];
        }
      }
    // dW4^T [64 in][16 out] -> dW4 [3][64]
    tc::ld16(lane_addr + kTcDW4, v);
    if (m >= 0)
      for (int k = 0; k < 3; ++k) gp[off_w(4) + k * 64 + m] = v[k];
  } else {
    for (int i = tid; i < kNW + 4 * 64; i += blockDim.x) gp[i] = 0.f;
  }
  // the output bias gradients and the losses of the warps, summed in warp order (deterministic)
  if (tid < 3) gp[off_b(4) + tid] = have ? ((db4[tid] + db4[4 + tid]) + db4[8 + tid]) + db4[12 + tid] : 0.f;
  {
    float ls = warp_sum(loss_acc);
    if (lane == 0) s_loss[warp] = ls;
    __syncthreads();
    if (tid == 0) gp[kNP] = have ? ((s_loss[0] + s_loss[1]) + s_loss[2]) + s_loss[3] : 0.f;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::dealloc(tmem, kTrainTmemCols);
#undef RTB_WAIT
}

// ---------------------------------------------------------------------------
// Adam on the FP32 master parameters, then the BF16 copies; clears the
// gradient for the next step.
// ---------------------------------------------------------------------------
// The gradient (and, at kNP, the loss) is the sum of the training CTAs'
// rows, in CTA order; it stays in g for inspection.
__global__ void k_nrc_adam(float* __restrict__ w, const float* __restrict__ gpart, int n_part, float* __restrict__ g,
                           float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                           float c1, float c2, int apply) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > kNP) return;
  float gi = 0.f;
  for (int c = 0; c < n_part; ++c) gi += gpart[(size_t)c * kGPRow + i];
  g[i] = gi;
  if (i < kNP && apply) {
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void k_nrc_pack(const float* __restrict__ w, uint16_t* __restrict__ packed) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  float* pb = (float*)(packed + kPackedBf16);
  if (i < kPackedBf16) {
    float x = 0.f;
    if (i < kPW4) {   // W0..W3 [out][in]
      x = w[i];
    } else if (i < kPT1) {   // W4 padded to 16 rows
      int r = (i - kPW4) / 64, c = (i - kPW4) % 64;
      x = r < 3 ? w[off_w(4) + r * 64 + c] : 0.f;
    } else if (i < kPT4) {   // W1^T .. W3^T [in][out]
      int l = 1 + (i - kPT1) / 4096, j = (i - kPT1) % 4096;
      int in = j / 64, out = j % 64;
      x = w[off_w(l) + out * 64 + in];
    } else {   // W4^T [64 in][16 out]
      int in = (i - kPT4) / 16, out = (i - kPT4) % 16;
      x = out < 3 ? w[off_w(4) + out * 64 + in] : 0.f;
    }
    packed[i] = bf16_bits(x);
  } else if (i < kPackedBf16 + kPackedBias) {
    int j = i - kPackedBf16;
    pb[j] = j < 256 ? w[kNW + j] : (j < 259 ? w[kNW + j] : 0.f);
  }
}

__global__ void k_make_records(const float* __restrict__ pnv, int64_t n, float4* __restrict__ recs, int stride) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* q = pnv + 9 * i;
  float4* r = recs + stride * i;
  r[0] = make_float4(q[0], q[1], q[2], __int_as_float((int)i));
  r[1] = make_float4(q[3], q[4], q[5], 0.f);
  r[2] = make_float4(q[6], q[7], q[8], 0.f);
  if (stride == 4) r[3] = make_float4(1.f, 1.f, 1.f, 0.f);
}

void nrc_make_records(const float* pnv, const float* targets, int64_t n, float4* recs, int stride, cudaStream_t st) {
  (void)targets;
  k_make_records<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pnv, n, recs, stride);
}

}  // namespace rtb

// ---------------------------------------------------------------------------
// host API
// ---------------------------------------------------------------------------
using namespace rtb;

struct rt_nrc {
  const rt_scene* scene = nullptr;   // the scene it was created for (its box normalises the encoding)
  rt_nrc_config cfg;
  NrcDevice nd;
  Buf params, m, v, grad, packed;
  Buf gpart;   // the training CTAs' gradient rows (sm_count x kGPRow floats)
  Buf infer_q, train_q, train_target, counters;   // frame queues (render integration)
  int64_t infer_cap = 0, train_cap = 0;
  int64_t step = 0;
  uint64_t frame = 0;
  int sm_count = 0, infer_blocks = 0;
  float last_loss = 0.f;
};

namespace rtb {

static uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static bool g_smem_attr_set = false;

static rt_status nrc_setup_kernels() {
  if (g_smem_attr_set) return RT_OK;
  cudaError_t e = cudaFuncSetAttribute(k_nrc_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, kInferSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_nrc_train, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrainSmem);
  if (e != cudaSuccess) return cuda_error(e, "nrc kernel attributes");
  g_smem_attr_set = true;
  return RT_OK;
}

static rt_status nrc_pack(rt_nrc* r, cudaStream_t st) {
  int n = kPackedBf16 + kPackedBias;
  k_nrc_pack<<<(n + 255) / 256, 256, 0, st>>>((const float*)r->params.p, (uint16_t*)r->packed.p);
  return cuda_error(cudaGetLastError(), "nrc pack");
}

rt_status nrc_infer_launch(rt_nrc* r, const float4* recs, const unsigned* count, unsigned cap, float* fb,
                           float* out3, unsigned* status, cudaStream_t st, float* const* fbs) {
  rt_status rs = nrc_setup_kernels();
  if (rs) return rs;
  int blocks = r->infer_blocks;
  k_nrc_infer<<<blocks, kInferThreads, kInferSmem, st>>>(r->nd, recs, count, cap, fb, out3, status, fbs);
  return cuda_error(cudaGetLastError(), "nrc infer");
}

rt_status nrc_train_launch(rt_nrc* r, const float4* recs, const float* targets, const unsigned* count, unsigned cap,
                           unsigned* status, cudaStream_t st) {
  rt_status rs = nrc_setup_kernels();
  if (rs) return rs;
  if ((rs = ensure(r->gpart, (size_t)r->sm_count * kGPRow * sizeof(float)))) return rs;
  k_nrc_train<<<r->sm_count, kTrainThreads, kTrainSmem, st>>>(r->nd, recs, targets, count, cap, (float*)r->gpart.p,
                                                               status);
  r->step++;
  float c1 = 1.f - powf(r->cfg.beta1, (float)r->step), c2 = 1.f - powf(r->cfg.beta2, (float)r->step);
  k_nrc_adam<<<(kNP + 1 + 255) / 256, 256, 0, st>>>((float*)r->params.p, (const float*)r->gpart.p, r->sm_count,
                                                     (float*)r->grad.p, (float*)r->m.p, (float*)r->v.p, r->cfg.lr,
                                                     r->cfg.beta1, r->cfg.beta2, r->cfg.eps, c1, c2, 1);
  rs = nrc_pack(r, st);
  if (rs) return rs;
  return cuda_error(cudaGetLastError(), "nrc train");
}

NrcDevice* nrc_device(rt_nrc* r) { return &r->nd; }

const rt_scene* nrc_scene(const rt_nrc* r) { return r->scene; }

const unsigned* nrc_prev_hits(rt_nrc* r) { return (const unsigned*)r->counters.p + 4; }

void nrc_keep_hits(rt_nrc* r, const unsigned* hits, cudaStream_t st) {
  cudaMemcpyAsync((unsigned*)r->counters.p + 4, hits, 4, cudaMemcpyDeviceToDevice, st);
}

rt_status nrc_frame_buffers(rt_nrc* r, int64_t ray_cap, bool train, NrcFrame* out) {
  int64_t icap = std::max<int64_t>(ray_cap, 65536);
  int64_t tcap = r->cfg.train_batch;
  rt_status rs;
  bool fresh = !r->counters.p;
  if ((rs = ensure(r->infer_q, (size_t)icap * 64)) || (rs = ensure(r->train_q, (size_t)tcap * 48)) ||
      (rs = ensure(r->train_target, (size_t)tcap * 12)) || (rs = ensure(r->counters, 64)))
    return rs;
  if (fresh) cudaMemset(r->counters.p, 0, 64);
  r->frame++;
  uint64_t sd = r->cfg.seed ^ (r->frame * 0x9E3779B97F4A7C15ull);
  out->depth = r->cfg.terminate_depth;
  out->target = (float*)r->train_target.p;
  out->infer_q = (float4*)r->infer_q.p;
  out->train_q = (float4*)r->train_q.p;
  out->infer_cap = (unsigned)icap;
  out->train_cap = (unsigned)tcap;
  out->train_batch = (unsigned)tcap;
  out->seed = (uint32_t)(splitmix64(sd) >> 32);
  r->nd.target = out->target;
  (void)train;
  return RT_OK;
}

}  // namespace rtb

extern "C" {

void rt_nrc_config_default(rt_nrc_config* c) {
  if (!c) return;
  c->train_batch = 65536;
  c->terminate_depth = 2;
  c->lr = 1e-2f;
  c->beta1 = 0.9f;
  c->beta2 = 0.99f;
  c->eps = 1e-8f;
  c->seed = 1;
}

rt_status rt_nrc_create(rt_scene* s, const rt_nrc_config* cfg_in, rt_nrc** out) {
  if (!s || !out) return set_error(RT_ERR_INVALID_ARG, "rt_nrc_create: NULL argument");
  *out = nullptr;
  rt_nrc_config cfg;
  rt_nrc_config_default(&cfg);
  if (cfg_in) cfg = *cfg_in;
  if (cfg.train_batch < 128 || cfg.train_batch > (1 << 22) || cfg.terminate_depth < 1 ||
      cfg.terminate_depth > RT_MAX_DEPTH || !(cfg.lr > 0.f) || !(cfg.beta1 >= 0.f && cfg.beta1 < 1.f) ||
      !(cfg.beta2 >= 0.f && cfg.beta2 < 1.f) || !(cfg.eps > 0.f))
    return set_error(RT_ERR_INVALID_ARG, "rt_nrc_create: invalid configuration");
  rt_nrc* r = new rt_nrc();
  r->scene = s;
  r->cfg = cfg;
  cudaDeviceGetAttribute(&r->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  r->infer_blocks = r->sm_count * 2;
  for (int j = 0; j < 3; ++j) {
    float lo = s->bbox_lo[j], hi = s->bbox_hi[j];
    if (!(hi > lo)) hi = lo + 1.f;
    r->nd.lo[j] = lo;
    r->nd.inv_ext[j] = 1.f / (hi - lo);
  }
  rt_status rs;
  if ((rs = ensure(r->params, kNP * 4)) || (rs = ensure(r->m, kNP * 4)) || (rs = ensure(r->v, kNP * 4)) ||
      (rs = ensure(r->grad, (kNP + 16) * 4)) || (rs = ensure(r->packed, kPackedBytes))) {
    rt_nrc_destroy(r);
    return rs;
  }
  // He-uniform initialisation, seeded; biases zero
  std::vector<float> w(kNP, 0.f);
  uint64_t st = cfg.seed * 0x2545F4914F6CDD1Dull + 12345;
  for (int l = 0; l < 5; ++l) {
    int fan_in = l == 0 ? kFeatures : 64;
    float a = std::sqrt(6.0f / (float)fan_in);
    for (int o = 0; o < d_out(l); ++o)
      for (int i = 0; i < d_in(l); ++i) {
        float u = (float)((splitmix64(st) >> 11) * (1.0 / 9007199254740992.0));
        w[off_w(l) + o * d_in(l) + i] = (l == 0 && i >= kFeatures) ? 0.f : (2.f * u - 1.f) * a;
      }
  }
  cudaError_t e = cudaMemcpy(r->params.p, w.data(), kNP * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(r->m.p, 0, kNP * 4);
  if (e == cudaSuccess) e = cudaMemset(r->v.p, 0, kNP * 4);
  if (e != cudaSuccess) {
    rt_nrc_destroy(r);
    return cuda_error(e, "rt_nrc_create");
  }
  if ((rs = ensure(r->counters, 64)) != RT_OK || cudaMemset(r->counters.p, 0, 64) != cudaSuccess) {
    rt_nrc_destroy(r);
    return rs ? rs : set_error(RT_ERR_CUDA, "rt_nrc_create: memset");
  }
  r->nd.packed = r->packed.p;
  r->nd.target = nullptr;
  if ((rs = nrc_pack(r, 0)) || (rs = nrc_setup_kernels())) {
    rt_nrc_destroy(r);
    return rs;
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    rt_nrc_destroy(r);
    return cuda_error(e, "rt_nrc_create");
  }
  *out = r;
  return RT_OK;
}

rt_status rt_nrc_destroy(rt_nrc* r) {
  if (!r) return RT_OK;
  cudaDeviceSynchronize();
  release(r->params);
  release(r->m);
  release(r->v);
  release(r->grad);
  release(r->gpart);
  release(r->packed);
  release(r->infer_q);
  release(r->train_q);
  release(r->train_target);
  release(r->counters);
  delete r;
  return RT_OK;
}

rt_status rt_nrc_get_params(rt_nrc* r, float* host, void* stream) {
  if (!r || !host) return set_error(RT_ERR_INVALID_ARG, "rt_nrc_get_params: NULL argument");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemcpy(host, r->params.p, kNP * 4, cudaMemcpyDeviceToHost);
  return cuda_error(e, "rt_nrc_get_params");
}

// File layout of rt_nrc_save: header, then params, m, v (kNP floats each).
struct NrcFileHeader {
  char magic[8];          // "RTBNRC" 0 1
  uint32_t version;       // 1
  uint32_t n_params;      // kNP
  rt_nrc_config cfg;
  int64_t step;
};
static const char kNrcMagic[8] = {'R', 'T', 'B', 'N', 'R', 'C', 0, 1};

rt_status rt_nrc_save(rt_nrc* r, const char* path, void* stream) {
  if (!r || !path) return set_error(RT_ERR_INVALID_ARG, "rt_nrc_save: NULL argument");
  std::vector<float> buf(3 * (size_t)kNP);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemcpy(buf.data(), r->params.p, kNP * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(buf.data() + kNP, r->m.p, kNP * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(buf.data() + 2 * kNP, r->v.p, kNP * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "rt_nrc_save");
  NrcFileHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kNrcMagic, 8);
  h.version = 1;
  h.n_params = kNP;
  h.cfg = r->cfg;
  h.step = r->step;
  FILE* f = fopen(path, "wb");
  if (!f) return set_error(RT_ERR_INVALID_ARG, std::string("rt_nrc_save: cannot open ") + path);
  bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(buf.data(), 4, buf.size(), f) == buf.size();
  ok = (fclose(f) == 0) && ok;
  if (!ok) return set_error(RT_ERR_INVALID_ARG, std::string("rt_nrc_save: cannot write ") + path);
  return RT_OK;
}

rt_status rt_nrc_load(rt_nrc* r, const char* path, void* stream) {
  if (!r || !path) return set_error(RT_ERR_INVALID_ARG, "rt_nrc_load: NULL argument");
  FILE* f = fopen(path, "rb");
  if (!f) return set_error(RT_ERR_INVALID_ARG, std::string("rt_nrc_load: cannot open ") + path);
  NrcFileHeader h;
  std::vector<float> buf(3 * (size_t)kNP);
  bool ok = fread(&h, sizeof(h), 1, f) == 1 && fread(buf.data(), 4, buf.size(), f) == buf.size();
  char extra;
  ok = ok && fread(&extra, 1, 1, f) == 0;   // nothing after the arrays
  fclose(f);
  if (!ok) return set_error(RT_ERR_INVALID_ARG, "rt_nrc_load: truncated file or trailing bytes");
  if (memcmp(h.magic, kNrcMagic, 8) != 0 || h.version != 1 || h.n_params != (uint32_t)kNP)
    return set_error(RT_ERR_INVALID_ARG, "rt_nrc_load: not a radiance-cache file of this format");
  const rt_nrc_config& c = h.cfg;
  if (c.train_batch < 1 || c.terminate_depth < 0 || c.terminate_depth > RT_MAX_DEPTH || !std::isfinite(c.lr) ||
      !std::isfinite(c.beta1) || !std::isfinite(c.beta2) || !std::isfinite(c.eps) || h.step < 0)
    return set_error(RT_ERR_INVALID_ARG, "rt_nrc_load: invalid configuration");
  for (float x : buf)
    if (!std::isfinite(x)) return set_error(RT_ERR_INVALID_ARG, "rt_nrc_load: non-finite value");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(r->params.p, buf.data(), kNP * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r->m.p, buf.data() + kNP, kNP * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r->v.p, buf.data() + 2 * kNP, kNP * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_error(e, "rt_nrc_load");
  r->cfg = c;
  r->step = h.step;
  return nrc_pack(r, st);
}

rt_status rt_nrc_set_params(rt_nrc* r, const float* host, void* stream) {
  if (!r || !host) return set_error(RT_ERR_INVALID_ARG, "rt_nrc_set_params: NULL argument");
  for (int i = 0; i < kNP; ++i)
    if (!std::isfinite(host[i])) return set_error(RT_ERR_INVALID_ARG, "rt_nrc_set_params: non-finite value");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(r->params.p, host, kNP * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(r->m.p, 0, kNP * 4);
  if (e == cudaSuccess) e = cudaMemset(r->v.p, 0, kNP * 4);
  if (e != cudaSuccess) return cuda_error(e, "rt_nrc_set_params");
  r->step = 0;
  return nrc_pack(r, st);
}

rt_status rt_nrc_get_grads(rt_nrc* r, float* host, float* loss, void* stream) {
  if (!r || !host) return set_error(RT_ERR_INVALID_ARG, "rt_nrc_get_grads: NULL argument");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemcpy(host, r->grad.p, kNP * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && loss) e = cudaMemcpy(loss, (float*)r->grad.p + kNP, 4, cudaMemcpyDeviceToHost);
  return cuda_error(e, "rt_nrc_get_grads");
}

// Plain queries (tests, tools): n hits (p, n, v) -> radiance exp(MLP).
rt_status rt_nrc_infer(rt_nrc* r, rt_scene* s, const float* pnv_dev, int64_t n, float* out_dev, void* stream) {
  if (!r || !s || (n > 0 && (!pnv_dev || !out_dev)) || n < 0 || n > (1 << 26))
    return set_error(RT_ERR_INVALID_ARG, "rt_nrc_infer: bad argument");
  if (n == 0) return RT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  rt_status rs;
  if ((rs = ensure(r->infer_q, (size_t)n * 64)) || (rs = ensure(r->counters, 64))) return rs;
  cudaError_t e = cudaMemcpyAsync(r->counters.p, &n, 4, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "rt_nrc_infer");
  nrc_make_records(pnv_dev, nullptr, n, (float4*)r->infer_q.p, 4, st);
  return nrc_infer_launch(r, (const float4*)r->infer_q.p, (const unsigned*)r->counters.p, (unsigned)n, nullptr,
                          out_dev, s->status, st);
}

// One training step on n given samples (p, n, v) with targets (n x 3):
// gradients (rt_nrc_get_grads), then Adam.
rt_status rt_nrc_train_step(rt_nrc* r, rt_scene* s, const float* pnv_dev, const float* target_dev, int64_t n,
                            void* stream) {
  if (!r || !s || n <= 0 || n > (1 << 26) || !pnv_dev || !target_dev)
    return set_error(RT_ERR_INVALID_ARG, "rt_nrc_train_step: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  rt_status rs;
  if ((rs = ensure(r->train_q, (size_t)n * 48)) || (rs = ensure(r->counters, 64))) return rs;
  cudaError_t e = cudaMemcpyAsync((unsigned*)r->counters.p + 1, &n, 4, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "rt_nrc_train_step");
  nrc_make_records(pnv_dev, target_dev, n, (float4*)r->train_q.p, 3, st);
  return nrc_train_launch(r, (const float4*)r->train_q.p, target_dev, (const unsigned*)r->counters.p + 1,
                          (unsigned)n, s->status, st);
}

}  // extern "C"
