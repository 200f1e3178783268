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

#include <cooperative_groups.h>

#include "nrc_internal.cuh"
#include "rtb_internal.cuh"
#include "tc.cuh"

namespace cg = cooperative_groups;

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

// The packed copy the kernels read: the BF16 weights as the shared-memory
// image of the forward operands (W_l as [out][in] in the K-major core-matrix
// layout of tc::core_off; W4 padded to 16 rows of zeros), so that one bulk
// copy stages them, then the FP32 biases (b0..b3, b4 padded to 16).  The
// backward pass reads the same tiles as MN-major operands: W_l^T needs no
// copy of its own.
constexpr int kImgW0 = 0, kImgW1 = 12288, kImgW2 = 20480, kImgW3 = 28672, kImgW4 = 36864;   // bytes
constexpr int kImgBytes = 38912;
constexpr int kPackedBias = 4 * 64 + 16;
constexpr int kPackedBytes = kImgBytes + kPackedBias * 4;   // 40,000
__host__ __device__ constexpr int img_off(int l) {
  return l == 0 ? kImgW0 : l == 1 ? kImgW1 : l == 2 ? kImgW2 : l == 3 ? kImgW3 : kImgW4;
}
static_assert(kImgBytes % 16 == 0 && kPackedBytes % 16 == 0, "bulk copies move whole 16-byte units");

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_float(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// ---------------------------------------------------------------------------
// encoding: 3 normalised position values, normal (3), view direction (3),
// sin and cos of 2^k pi x_hat_j for k = 0..11 -> 81 values, zero-padded to 96
// ---------------------------------------------------------------------------

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

// The 96 features of one sample (p, n, v) as row t of a K-major [128][96]
// tile, each 16-byte chunk stored as soon as its 8 features exist (fewer
// live registers than encoding the whole row first).  A row past the batch
// is zero.  With ones81 the first padding column (feature 81) of a sample
// is 1: the layer-0 weight-gradient MMA then also sums the backward signal
// over the batch (dB0), against a weight column the packed copy keeps 0.
__device__ __forceinline__ void encode_store(const float* pnv, const float* lo, const float* inv_ext, bool valid,
                                             uint8_t* tile, int t, bool ones81 = false) {
  float f[96];
  float xh[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    xh[j] = (pnv[j] - lo[j]) * inv_ext[j];
    f[j] = valid ? xh[j] : 0.f;
    f[3 + j] = valid ? pnv[3 + j] : 0.f;
    f[6 + j] = valid ? pnv[6 + j] : 0.f;
  }
  store_chunk(tile, t, 0, 96, f);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float sc = (float)(1 << k);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float sn, cs;
      sincospif(sc * xh[j], &sn, &cs);
      f[9 + 6 * k + j] = valid ? sn : 0.f;
      f[9 + 6 * k + 3 + j] = valid ? cs : 0.f;
    }
    const int have = 9 + 6 * (k + 1);   // features formed so far
#pragma unroll
    for (int c = 1; c < 10; ++c)
      if (8 * c + 8 <= have && 8 * c + 8 > have - 6) store_chunk(tile, t, c, 96, f + 8 * c);
  }
#pragma unroll
  for (int k = kFeatures; k < 96; ++k) f[k] = 0.f;
  if (ones81 && valid) f[kFeatures] = 1.f;
  store_chunk(tile, t, 10, 96, f + 80);
  store_chunk(tile, t, 11, 96, f + 88);
}

// ---------------------------------------------------------------------------
// inference: records (p, n, v, weight, pixel) -> pixel += weight * exp(MLP)
// 128 threads, one sample per thread, one 128-sample tile at a time.
// ---------------------------------------------------------------------------
constexpr int kInferThreads = 128;
constexpr int kInferTmemCols = 64;
// dynamic shared memory (bytes), 1 KB aligned sections
constexpr int kSmW0 = kImgW0, kSmW1 = kImgW1, kSmW2 = kImgW2, kSmW3 = kImgW3, kSmW4 = kImgW4;
constexpr int kSmBias = kImgBytes;   // 272 floats: the packed copy lands here whole
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
                                                            const float* __restrict__ pnv,
                                                            const unsigned* __restrict__ count, unsigned cap,
                                                            float* __restrict__ fb, float* __restrict__ out3,
                                                            unsigned* status, float* const* __restrict__ fbs) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* mbar = (uint64_t*)(sm + kSmMisc);
  uint32_t* tslot = (uint32_t*)(sm + kSmMisc + 8);
  int* abort_flag = (int*)(sm + kSmMisc + 16);
  float* bias = (float*)(sm + kSmBias);
  int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t wbar = tc::smem_u32(sm + kSmMisc + 24);
  // a CTA without a tile returns before staging anything
  const unsigned n = count ? min(*count, cap) : cap;
  if (blockIdx.x >= (n + 127) / 128) return;
  if (warp == 0) tc::alloc(tc::smem_u32(tslot), kInferTmemCols);
  if (tid == 0) {
    tc::mbar_init(tc::smem_u32(mbar), 1);
    tc::mbar_init(wbar, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    // the weights' shared-memory image and the biases: one bulk copy
    tc::mbar_expect_tx(wbar, kPackedBytes);
    tc::bulk_g2s(tc::smem_u32(sm), nd.packed, kPackedBytes, wbar);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const bool w_ok = !__syncthreads_or(!tc::mbar_wait(wbar, 0));
  if (!w_ok && tid == 0) atomicOr(status, kErrNrcTimeout);
  uint32_t tmem = *tslot;
  uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t mb = tc::smem_u32(mbar);
  uint32_t sA = tc::smem_u32(sm + kSmA);
  const uint32_t sW[5] = {tc::smem_u32(sm + kSmW0), tc::smem_u32(sm + kSmW1), tc::smem_u32(sm + kSmW2),
                          tc::smem_u32(sm + kSmW3), tc::smem_u32(sm + kSmW4)};
  unsigned tiles = w_ok ? (n + 127) / 128 : 0u;
  uint32_t phase = 0;
  float lo[3] = {nd.lo[0], nd.lo[1], nd.lo[2]}, ie[3] = {nd.inv_ext[0], nd.inv_ext[1], nd.inv_ext[2]};
  // a query's inputs: position, normal, direction (q[0..8]), frame (q[9]);
  // path weight and pixel (w)
  auto fetch = [&](unsigned tl, float* q, float4& w) {
    const unsigned row = tl * 128 + tid;
    if (tl >= tiles || row >= n) return;
    if (pnv) {
      // caller arrays: p, n, v of query `row`, weight 1 (outputs to out3 only)
#pragma unroll
      for (int j = 0; j < 9; ++j) q[j] = pnv[9 * (size_t)row + j];
      w = make_float4(1.f, 1.f, 1.f, 0.f);
    } else {
      const float4 q0 = recs[4 * (size_t)row], q1 = recs[4 * (size_t)row + 1], q2 = recs[4 * (size_t)row + 2],
                   q3 = recs[4 * (size_t)row + 3];
      q[0] = q0.x, q[1] = q0.y, q[2] = q0.z, q[3] = q1.x, q[4] = q1.y, q[5] = q1.z, q[6] = q2.x, q[7] = q2.y;
      q[8] = q2.z;
      q[9] = q3.w;
      w = make_float4(q3.x, q3.y, q3.z, q0.w);
    }
  };
  float nq[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float4 nw = make_float4(0.f, 0.f, 0.f, 0.f);
  fetch(blockIdx.x, nq, nw);
  for (unsigned tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    unsigned row = tile * 128 + tid;
    bool valid = row < n;
    float q[10];
#pragma unroll
    for (int j = 0; j < 10; ++j) q[j] = nq[j];
    const float wr = nw.x, wg = nw.y, wb = nw.z;
    const int pixel = __float_as_int(nw.w), frame = __float_as_int(q[9]);
    // the next tile's inputs load while this one runs
    fetch(tile + gridDim.x, nq, nw);
    encode_store(q, lo, ie, valid, sm + kSmA, tid);
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
// the packed copy
// ---------------------------------------------------------------------------
// Writes parameter i (oracle layout) into the packed copy.
__device__ __forceinline__ void pack_param(uint8_t* __restrict__ packed, int i, float x) {
  if (i < kNW) {
    const int l = i < off_w(1) ? 0 : min(1 + (i - off_w(1)) / 4096, 4);
    const int rel = i - off_w(l), o = rel / d_in(l), c = rel % d_in(l);
    // the padding features' weights stay 0: the training encoding puts a 1 in feature 81
    *(uint16_t*)(packed + img_off(l) + tc::core_off(o, c, d_in(l))) = (l == 0 && c >= kFeatures) ? 0 : bf16_bits(x);
  } else {
    ((float*)(packed + kImgBytes))[i - kNW] = x;   // b0..b3 (64 each), then b4 (3)
  }
}

// Every parameter into a zeroed packed copy (creation, loading).
__global__ void k_nrc_pack(const float* __restrict__ w, uint8_t* __restrict__ packed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kNP) pack_param(packed, i, w[i]);
}

// ---------------------------------------------------------------------------
// training: forward (activations kept), loss gradient, backward; weight and
// bias gradients accumulate in tensor memory over the CTA's tiles, then go
// to its own row of the gradient buffer.  One CTA per SM (its 512
// tensor-memory columns) keeps two tiles of 128 samples in flight: warpgroup
// s (warps 4s..4s+3, one sample a thread) runs the epilogues of the tiles of
// slot s, and one lane of warp 8 issues every MMA, alternating between the
// slots stage by stage in a fixed order.  One slot's epilogue runs while the
// other slot's MMAs do, and the accumulated gradient does not depend on
// timing.
//
// Every activation is stored once, row by row (a sample's features in
// 16-byte chunks, the K-major layout of the forward MMAs).  The
// weight-gradient MMAs, whose K is the batch, read the same tiles as
// MN-major operands, and the backward MMAs read the forward weight tiles as
// MN-major W^T, so no transposed copy is made.  The backward signal dZ_l
// is written over H_l once dW_l has been formed from H_l.  The bias
// gradients are MMAs of dZ^T against a block of ones (one K = 16 step's
// operand, read again at every step).
// ---------------------------------------------------------------------------
constexpr int kTrainWarps = 9;   // two epilogue warpgroups, then the MMA warp
constexpr int kTrainThreads = 32 * kTrainWarps;
constexpr int kTrainTmemCols = 512;
// tensor-memory columns (16-aligned)
constexpr int kTcAcc = 0;      // 64 a slot, at 64 s: forward / backward accumulator (M = 128)
constexpr int kTcDW0 = 128;    // 96: dW0 (M = 64 out, N = 96 in)
constexpr int kTcDW1 = 224;    // 64 each at 224, 288, 352: dW1..dW3
constexpr int kTcDW4 = 416;    // 16: dW4^T (M = 64 in, N = 16 out)
constexpr int kTcDB = 432;     // 16 each at 432 + 16 l: dB1..dB3 (M = 64 out; every column the same sum); dB0 is in dW0
static_assert(kTcDB + 4 * 16 <= kTrainTmemCols, "the training accumulators exceed the tensor memory");
__host__ __device__ constexpr int tc_dw(int l) { return l == 0 ? kTcDW0 : kTcDW1 + 64 * (l - 1); }
// shared memory (bytes): the weight image and the FP32 biases (one bulk
// copy of the packed buffer), a block of ones, control words, then two slots
constexpr int kTsBias = kImgBytes;         // 272 floats
constexpr int kTsOnes = kTsBias + kPackedBias * 4;   // [16][16] ones, K-major: 512 B
constexpr int kTsMisc = kTsOnes + 512;     // mbarriers, tensor-memory slot, abort flag, per-warp sums
constexpr int kTsSlot0 = kTsMisc + 256;
constexpr int kTsX = 0;                    // within a slot: X [128][96]
constexpr int kTsH = 24576;                // H1..H4 [128][64], 16 KB each (then dZ1..dZ4)
constexpr int kTsZ5 = kTsH + 4 * 16384;    // dZ5 [128][16]
constexpr int kTsSlotBytes = kTsZ5 + 4096;
constexpr int kTrainSmem = kTsSlot0 + 2 * kTsSlotBytes;
static_assert(kTrainSmem <= 227 * 1024, "the training CTA's shared memory exceeds the per-block limit");
static_assert(kTsSlot0 % 16 == 0 && kTsSlotBytes % 16 == 0, "operand tiles start on 16-byte boundaries");

// Bytes an operand read spans from its start address (one past the last
// byte), for the two unswizzled layouts the MMAs below use: K-major (8-row
// groups `sbo` apart, K = 16 steps 256 B apart) and MN-major (K = 16 steps
// 2 k_pitch apart, 8-element chunks along M or N 128 B apart).  Each
// operand's span must fit its tile: no MMA reads past it.
__host__ __device__ constexpr int span_kmajor(int rows, int K, int sbo) {
  return (rows / 8 - 1) * sbo + (K / 16 - 1) * 256 + 256;
}
__host__ __device__ constexpr int span_mnmajor(int mn, int K, int k_pitch) {
  return (K / 16 - 1) * 2 * k_pitch + k_pitch + (mn / 8 - 1) * 128 + 128;
}
static_assert(span_kmajor(128, 96, 1536) <= 24576 && span_kmajor(128, 64, 1024) <= 16384 &&
                  span_kmajor(128, 16, 256) <= 4096, "forward A operands (X, H_l, dZ5)");
static_assert(span_kmajor(64, 96, 1536) <= kImgW1 - kImgW0 && span_kmajor(64, 64, 1024) <= kImgW2 - kImgW1 &&
                  span_kmajor(16, 64, 1024) <= kImgBytes - kImgW4, "forward B operands (W_l)");
static_assert(span_mnmajor(64, 64, 1024) <= kImgW2 - kImgW1 && span_mnmajor(64, 16, 1024) <= kImgBytes - kImgW4,
              "backward B operands (W_l^T)");
static_assert(span_mnmajor(64, 128, 1024) <= 16384 && span_mnmajor(16, 128, 256) <= 4096 &&
                  span_mnmajor(96, 128, 1536) <= 24576 && span_kmajor(16, 16, 256) <= 512,
              "weight- and bias-gradient operands (H_l, dZ_l, dZ5, X, ones)");

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

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Waits for an mbarrier phase; gives up after ~2^14 suspended polls or once another
// thread of the CTA has raised the abort flag.
__device__ __forceinline__ bool train_wait(uint32_t mbar, uint32_t parity, volatile int* abort_flag) {
  // each poll suspends the thread for up to ~1 us; 2^14 of them bound the wait
  for (int i = 0; i < (1 << 14); ++i) {
    if (tc::mbar_try_wait_hint(mbar, parity, 1000u)) return true;
    if (*abort_flag) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// Issues NK back-to-back MMAs: step j reads A at a + j a_step and B at
// b + j b_step (bytes; the descriptors' start-address fields advance by
// step / 16, far from overflowing below 256 KB).
template <int NK>
__device__ __forceinline__ void mma_k(uint32_t d, uint64_t a, uint32_t a_step, uint64_t b, uint32_t b_step,
                                      uint32_t idesc, bool accumulate) {
#pragma unroll
  for (int j = 0; j < NK; ++j)
    tc::mma(d, a + (uint64_t)((a_step >> 4) * j), b + (uint64_t)((b_step >> 4) * j), idesc,
            (accumulate || j > 0) ? 1u : 0u);
}
// K-major operand (8-row groups sbo apart) and MN-major operand (8-row K
// groups k_pitch apart, 8-element chunks 128 B apart) descriptors.
__device__ __forceinline__ uint64_t kdesc(uint32_t a, uint32_t sbo) { return tc::smem_desc(a, 128u, sbo); }
__device__ __forceinline__ uint64_t mndesc(uint32_t a, uint32_t k_pitch) { return tc::smem_desc(a, k_pitch, 128u); }

// The MMAs of one stage of slot s (issued by one thread): stages 0..4 are
// the forward layers, 5..9 the backward layers 4..0.  `first` starts the
// gradient accumulators (the CTA's first tile).  sbase is the shared-memory
// address of the weight image (the start of the CTA's shared memory).
__device__ __noinline__ void train_issue(uint32_t sbase, uint32_t tmem, int s, int stage, bool first) {
  const uint32_t acc = tmem + kTcAcc + 64u * s;
  const uint32_t slot = sbase + kTsSlot0 + (uint32_t)s * kTsSlotBytes;
  const uint32_t X = slot + kTsX, Z5 = slot + kTsZ5, ones = sbase + kTsOnes;
  const uint32_t f128_64 = tc::idesc_bf16_f32(128, 64);
  switch (stage) {
    case 0:
      mma_k<6>(acc, kdesc(X, 1536u), 256u, kdesc(sbase + kImgW0, 1536u), 256u, f128_64, false);
      break;
    case 1:
    case 2:
    case 3:
      mma_k<4>(acc, kdesc(slot + kTsH + 16384u * (stage - 1), 1024u), 256u, kdesc(sbase + img_off(stage), 1024u),
               256u, f128_64, false);
      break;
    case 4:
      mma_k<4>(acc, kdesc(slot + kTsH + 3 * 16384u, 1024u), 256u, kdesc(sbase + kImgW4, 1024u), 256u,
               tc::idesc_bf16_f32(128, 16), false);
      break;
    case 5: {
      // dW4^T [64 in][16 out] += H4^T dZ5 (both MN-major over the batch)
      mma_k<8>(tmem + kTcDW4, mndesc(slot + kTsH + 3 * 16384u, 1024u), 2048u, mndesc(Z5, 256u), 512u,
               tc::idesc_bf16_f32_mn(64, 16), !first);
      // dH4 = dZ5 W4: A = dZ5 (K-major, K = 16), B = W4 read as W4^T (MN-major)
      tc::mma(acc, kdesc(Z5, 256u), mndesc(sbase + kImgW4, 1024u), tc::idesc_bf16_f32_bmn(128, 64), 0u);
      break;
    }
    default: {
      const int l = 9 - stage;   // 3, 2, 1, 0
      const uint32_t dz = slot + kTsH + 16384u * l;   // dZ_{l+1}, over H_{l+1}
      // dW_l [out][in] += dZ_{l+1}^T H_l, and dB_l += dZ_{l+1}^T 1 (layer 0: in dW0)
      if (l == 0)
        mma_k<8>(tmem + kTcDW0, mndesc(dz, 1024u), 2048u, mndesc(X, 1536u), 3072u, tc::idesc_bf16_f32_mn(64, 96),
                 !first);
      else
        mma_k<8>(tmem + tc_dw(l), mndesc(dz, 1024u), 2048u, mndesc(slot + kTsH + 16384u * (l - 1), 1024u), 2048u,
                 tc::idesc_bf16_f32_mn(64, 64), !first);
      if (l > 0)   // dB0 is column 81 of dW0 (the ones column of X)
        mma_k<8>(tmem + kTcDB + 16u * l, mndesc(dz, 1024u), 2048u, kdesc(ones, 256u), 0u,
                 tc::idesc_bf16_f32_amn(64, 16), !first);
      // dH_l = dZ_{l+1} W_l: A = dZ (K-major), B = W_l read as W_l^T (MN-major)
      if (l > 0)
        mma_k<4>(acc, kdesc(dz, 1024u), 256u, mndesc(sbase + img_off(l), 1024u), 2048u,
                 tc::idesc_bf16_f32_bmn(128, 64), false);
      break;
    }
  }
}

// A training sample's inputs: position, normal and direction, and its target.
__device__ __forceinline__ void train_fetch(const float4* __restrict__ recs, const float* __restrict__ pnv,
                                            const float* __restrict__ targets, unsigned row, bool valid, float* q,
                                            float* t3) {
  if (!valid) return;
  int slot;
  if (pnv) {
#pragma unroll
    for (int j = 0; j < 9; ++j) q[j] = pnv[9 * (size_t)row + j];
    slot = (int)row;
  } else {
    const float4 a = recs[3 * (size_t)row], b = recs[3 * (size_t)row + 1], c = recs[3 * (size_t)row + 2];
    q[0] = a.x, q[1] = a.y, q[2] = a.z, q[3] = b.x, q[4] = b.y, q[5] = b.z, q[6] = c.x, q[7] = c.y, q[8] = c.z;
    slot = __float_as_int(a.w);
  }
  t3[0] = targets[3 * (size_t)slot];
  t3[1] = targets[3 * (size_t)slot + 1];
  t3[2] = targets[3 * (size_t)slot + 2];
}

// The Adam step that follows the gradient in the same launch.
struct AdamStep {
  float *w, *g, *m, *v;   // FP32 masters, summed gradient (and loss at kNP), moments
  uint8_t* packed;        // the packed copy the kernels read
  float lr, b1, b2, eps, c1, c2;
  int apply;
};

__device__ __forceinline__ void adam_update(const AdamStep& a, int i, float gi) {
  a.g[i] = gi;
  if (i < kNP && a.apply) {
    const float mi = a.b1 * a.m[i] + (1.f - a.b1) * gi;
    const float vi = a.b2 * a.v[i] + (1.f - a.b2) * gi * gi;
    a.m[i] = mi;
    a.v[i] = vi;
    const float wi = a.w[i] - a.lr * (mi / a.c1) / (sqrtf(vi / a.c2) + a.eps);
    a.w[i] = wi;
    pack_param(a.packed, i, wi);
  }
}

// After every CTA has written its gradient row: this CTA's slice of the
// parameters (and the loss, the last entry) is summed over the rows and
// stepped.  Threads 0..255: parameter t % 128 of a 128-wide chunk, rows of
// parity t / 128 in row order, then the two halves in order (the sum does
// not depend on timing).
__device__ void adam_slice(const float* __restrict__ gpart, int rows, const AdamStep& a, float* part) {
  const int tid = threadIdx.x, G = (int)gridDim.x;
  const int per = (kNP + 1 + G - 1) / G, beg = min(kNP + 1, (int)blockIdx.x * per), end = min(kNP + 1, beg + per);
  for (int p0 = beg; p0 < end; p0 += 128) {
    const int i = p0 + (tid & 127), h = tid >> 7;
    float sum = 0.f;
    if (tid < 256) {
      constexpr int kBatch = 40;   // loads in flight a thread
      for (int c0 = h; c0 < rows; c0 += 2 * kBatch) {
        float r[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
          const int c = c0 + 2 * k;
          r[k] = (c < rows && i < end) ? __ldcg(&gpart[(size_t)c * kGPRow + i]) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k) sum += r[k];
      }
      part[tid] = sum;
    }
    __syncthreads();
    if (tid < 128 && i < end) adam_update(a, i, part[tid] + part[128 + tid]);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kTrainThreads, 1)
    k_nrc_train(NrcDevice nd, const float4* __restrict__ recs, const float* __restrict__ pnv,
                const float* __restrict__ targets, const unsigned* __restrict__ count, unsigned cap,
                float* __restrict__ gpart, unsigned* status, AdamStep adam) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const uint32_t full0 = tc::smem_u32(sm + kTsMisc), ready0 = full0 + 16, wbar = full0 + 32;
  uint32_t* tslot = (uint32_t*)(sm + kTsMisc + 40);
  volatile int* abort_flag = (volatile int*)(sm + kTsMisc + 44);
  float* s_loss = (float*)(sm + kTsMisc + 48);   // [8 warps]
  float* db4 = (float*)(sm + kTsMisc + 80);      // [8 warps][4]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::alloc(tc::smem_u32(tslot), kTrainTmemCols);
  if (tid == 32) {
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(full0 + 8 * s, 1);
      tc::mbar_init(ready0 + 8 * s, 4);   // one arrival a warp
    }
    tc::mbar_init(wbar, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    // the forward weights' shared-memory image and the biases: one bulk copy
    tc::mbar_expect_tx(wbar, kPackedBytes);
    tc::bulk_g2s(tc::smem_u32(sm), nd.packed, kPackedBytes, wbar);
  }
  {
    // the block of ones (BF16 1.0) and the per-warp sums
    uint4* o = (uint4*)(sm + kTsOnes);
    for (int i = tid; i < 512 / 16; i += blockDim.x) o[i] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
    if (tid < 32) db4[tid] = 0.f;
    if (tid < 8) s_loss[tid] = 0.f;
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const bool w_ok = !__syncthreads_or(!tc::mbar_wait(wbar, 0));
  if (!w_ok && tid == 0) atomicOr(status, kErrNrcTimeout);
  const uint32_t tmem = *tslot;
  const unsigned n = count ? min(*count, cap) : cap;
  const unsigned tiles = w_ok ? (n + 127) / 128 : 0u;
  const float* bias = (const float*)(sm + kTsBias);
  bool aborted = false;

  if (warp == 8) {
    // ---- the MMA issuer: stage by stage, slot 0 then slot 1 ----
    if (lane == 0 && tiles > 0) {
      const uint32_t sbase = tc::smem_u32(sm);
      uint32_t rph[2] = {0u, 0u};
      for (unsigned k = 0; !aborted && blockIdx.x + k * gridDim.x < tiles; k += 2) {
        const bool has1 = blockIdx.x + (k + 1) * gridDim.x < tiles;
        for (int stage = 0; stage < 10 && !aborted; ++stage)
          for (int s = 0; s < (has1 ? 2 : 1); ++s) {
            if (!train_wait(ready0 + 8 * s, rph[s], abort_flag)) {
              aborted = true;
              break;
            }
            rph[s] ^= 1u;
            tc::fence_after_sync();
            train_issue(sbase, tmem, s, stage, k == 0 && s == 0);
            tc::commit(full0 + 8 * s);
          }
      }
      if (aborted) {
        *abort_flag = 1;
        atomicOr(status, kErrNrcTimeout);
      }
    }
    __syncwarp();
  } else {
    // ---- the epilogues of slot s ----
    const int s = warp >> 2, t = tid & 127, wq = warp & 3;
    const uint32_t full = full0 + 8 * s, ready = ready0 + 8 * s;
    const uint32_t acc = tmem + ((uint32_t)(wq * 32) << 16) + kTcAcc + 64u * s;   // this warp's lane quarter
    uint8_t* slot = sm + kTsSlot0 + s * kTsSlotBytes;
    const float lo[3] = {nd.lo[0], nd.lo[1], nd.lo[2]}, ie[3] = {nd.inv_ext[0], nd.inv_ext[1], nd.inv_ext[2]};
    uint32_t fph = 0u;
    float loss_acc = 0.f;
    float q[9] = {}, tq[3] = {};
    unsigned tile = blockIdx.x + (unsigned)s * gridDim.x;
    train_fetch(recs, pnv, targets, tile * 128 + t, tile < tiles && tile * 128 + t < n, q, tq);
    for (; tile < tiles; tile += 2 * gridDim.x) {
      const unsigned row = tile * 128 + t;
      const bool valid = row < n;
      const float tr = tq[0], tg = tq[1], tb = tq[2];
      encode_store(q, lo, ie, valid, slot + kTsX, t, true);
      // the next tile of this slot: its inputs load while this one runs
      {
        const unsigned nt = tile + 2 * gridDim.x;
        train_fetch(recs, pnv, targets, nt * 128 + t, nt < tiles && nt * 128 + t < n, q, tq);
      }
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(ready);
      // forward epilogues: H_{l+1} = relu(Z_{l+1} + b_l), its ReLU mask kept
      uint32_t mask[4][2];
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        if (!train_wait(full, fph, abort_flag)) aborted = true;
        fph ^= 1u;
        tc::fence_after_sync();
        uint8_t* hl = slot + kTsH + 16384 * l;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          float h[32];
          tc::ld32(acc + 32 * half, h);
          const float4* b4 = (const float4*)(bias + 64 * l + 32 * half);
          uint32_t mk = 0u;
#pragma unroll
          for (int k4 = 0; k4 < 8; ++k4) {
            const float4 b = b4[k4];
            const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int k = 4 * k4 + e;
              const float z = h[k] + bb[e];
              const bool pos = valid && z > 0.f;
              mk |= (pos ? 1u : 0u) << k;
              h[k] = pos ? z : 0.f;
            }
          }
          // kept as an opaque word: otherwise the compiler carries the 64 ReLU
          // predicates of every layer to the backward pass in registers
          asm volatile("mov.b32 %0, %1;" : "=r"(mask[l][half]) : "r"(mk));
#pragma unroll
          for (int c = 0; c < 4; ++c) store_chunk(hl, t, 4 * half + c, 64, h + 8 * c);
        }
        tc::fence_before_sync();
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(ready);
      }
      // loss gradient at the exp output: dL/dz5 = 2 (y - t) / (y^2 + 0.01) / (3n) * y,
      // stored in BF16; the output bias gradient sums the stored values
      {
        if (!train_wait(full, fph, abort_flag)) aborted = true;
        fph ^= 1u;
        tc::fence_after_sync();
        float o[16];
        tc::ld16(acc, o);
        tc::fence_before_sync();
        const float inv_n3 = 1.0f / (3.0f * (float)n);
        float g[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) g[k] = 0.f;
        if (valid) {
          const float t3[3] = {tr, tg, tb};
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float y = expf(o[c] + bias[256 + c]);
            const float den = y * y + 0.01f;
            const float dy = y - t3[c];
            loss_acc += dy * dy / den * inv_n3;
            g[c] = 2.f * dy / den * inv_n3 * y;
          }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float sum = warp_sum(bf16_float(bf16_bits(g[c])));
          if (lane == 0) db4[4 * warp + c] += sum;
        }
        store_chunk(slot + kTsZ5, t, 0, 16, g);
        store_chunk(slot + kTsZ5, t, 1, 16, g + 8);
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(ready);
      }
      // backward epilogues: dZ_l = dH_l * relu'(z_l), stored over H_l
#pragma unroll
      for (int l = 4; l >= 1; --l) {
        if (!train_wait(full, fph, abort_flag)) aborted = true;
        fph ^= 1u;
        tc::fence_after_sync();
        uint8_t* hl = slot + kTsH + 16384 * (l - 1);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          float g[32];
          tc::ld32(acc + 32 * half, g);
          const uint32_t mk = mask[l - 1][half];
#pragma unroll
          for (int k = 0; k < 32; ++k) g[k] = ((mk >> k) & 1u) ? g[k] : 0.f;
#pragma unroll
          for (int c = 0; c < 4; ++c) store_chunk(hl, t, 4 * half + c, 64, g + 8 * c);
        }
        tc::fence_before_sync();
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(ready);
      }
      // the tile's last MMAs (dW0, dB0) read X and dZ1: done before the next tile overwrites them
      if (!train_wait(full, fph, abort_flag)) aborted = true;
      fph ^= 1u;
      tc::fence_after_sync();
      if (aborted) break;
    }
    if (aborted) {
      *abort_flag = 1;
      atomicOr(status, kErrNrcTimeout);
    }
    const float ls = warp_sum(loss_acc);
    if (lane == 0) s_loss[warp] = ls;
  }
  tc::fence_before_sync();
  aborted = __syncthreads_or(aborted) != 0;
  tc::fence_after_sync();

  // this CTA's gradients and loss: its own row of gpart (plain stores; the
  // Adam kernel sums the rows in a fixed order).  A CTA without a tile, or
  // one whose wait timed out, writes zeros.
  float* gp = gpart + (size_t)blockIdx.x * kGPRow;
  const bool have = !aborted && tiles > blockIdx.x;
  if (have && warp < 8) {
    // accumulator row m of an M = 64 MMA: lane (m / 16) * 32 + m % 16
    const int wq = warp & 3, m = wq * 16 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(wq * 32) << 16);
    const bool mine = lane < 16;
    float v[32];
    if (warp < 4) {
      for (int c = 0; c < 3; ++c) {   // dW0: 96 columns; column 81 is dB0, 81..95 are padding
        tc::ld32(lane_base + kTcDW0 + 32 * c, v);
        if (c == 2) {
          if (mine) gp[off_b(0) + m] = v[kFeatures - 64];
#pragma unroll
          for (int k = kFeatures - 64; k < 32; ++k) v[k] = 0.f;
        }
        if (mine) {
          store16(gp + off_w(0) + m * 96 + 32 * c, v);
          store16(gp + off_w(0) + m * 96 + 32 * c + 16, v + 16);
        }
      }
      for (int c = 0; c < 2; ++c) {   // dW1
        tc::ld32(lane_base + tc_dw(1) + 32 * c, v);
        if (mine) {
          store16(gp + off_w(1) + m * 64 + 32 * c, v);
          store16(gp + off_w(1) + m * 64 + 32 * c + 16, v + 16);
        }
      }
      tc::ld16(lane_base + kTcDB + 16, v);
      if (mine) gp[off_b(1) + m] = v[0];
    } else {
      for (int l = 2; l <= 3; ++l)
        for (int c = 0; c < 2; ++c) {
          tc::ld32(lane_base + tc_dw(l) + 32 * c, v);
          if (mine) {
            store16(gp + off_w(l) + m * 64 + 32 * c, v);
            store16(gp + off_w(l) + m * 64 + 32 * c + 16, v + 16);
          }
        }
      tc::ld16(lane_base + kTcDB + 32, v);
      if (mine) gp[off_b(2) + m] = v[0];
      tc::ld16(lane_base + kTcDB + 48, v);
      if (mine) gp[off_b(3) + m] = v[0];
      // dW4^T [64 in][16 out] -> dW4 [3][64]
      tc::ld16(lane_base + kTcDW4, v);
      if (mine)
        for (int k = 0; k < 3; ++k) gp[off_w(4) + k * 64 + m] = v[k];
    }
  } else if (!have) {
    for (int i = tid; i < kNW + 4 * 64; i += blockDim.x) gp[i] = 0.f;
  }
  // the output bias gradients and the losses of the warps, summed in warp order (deterministic)
  if (tid < 3) {
    float b = 0.f;
    for (int w8 = 0; w8 < 8; ++w8) b += db4[4 * w8 + tid];
    gp[off_b(4) + tid] = have ? b : 0.f;
  }
  if (tid == 0) {
    float l8 = 0.f;
    for (int w8 = 0; w8 < 8; ++w8) l8 += s_loss[w8];
    gp[kNP] = have ? l8 : 0.f;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::dealloc(tmem, kTrainTmemCols);
  // every CTA's row written (a cooperative launch: all CTAs are resident)
  cg::this_grid().sync();
  adam_slice(gpart, (int)gridDim.x, adam, (float*)(sm + kTsSlot0));
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
  if (e == cudaSuccess)   // the whole on-chip memory as shared memory: three inference CTAs an SM
    e = cudaFuncSetAttribute(k_nrc_infer, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_nrc_train, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrainSmem);
  if (e != cudaSuccess) return cuda_error(e, "nrc kernel attributes");
  g_smem_attr_set = true;
  return RT_OK;
}

static rt_status nrc_pack(rt_nrc* r, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(r->packed.p, 0, kPackedBytes, st);
  if (e != cudaSuccess) return cuda_error(e, "nrc pack");
  k_nrc_pack<<<(kNP + 255) / 256, 256, 0, st>>>((const float*)r->params.p, (uint8_t*)r->packed.p);
  return cuda_error(cudaGetLastError(), "nrc pack");
}

rt_status nrc_infer_launch(rt_nrc* r, const float4* recs, const unsigned* count, unsigned cap, float* fb,
                           float* out3, unsigned* status, cudaStream_t st, float* const* fbs, const float* pnv) {
  rt_status rs = nrc_setup_kernels();
  if (rs) return rs;
  int blocks = r->infer_blocks;
  k_nrc_infer<<<blocks, kInferThreads, kInferSmem, st>>>(r->nd, recs, pnv, count, cap, fb, out3, status, fbs);
  return cuda_error(cudaGetLastError(), "nrc infer");
}

rt_status nrc_train_launch(rt_nrc* r, const float4* recs, const float* targets, const unsigned* count, unsigned cap,
                           unsigned* status, cudaStream_t st, const float* pnv) {
  rt_status rs = nrc_setup_kernels();
  if (rs) return rs;
  if ((rs = ensure(r->gpart, (size_t)r->sm_count * kGPRow * sizeof(float)))) return rs;
  r->step++;
  AdamStep ad;
  ad.w = (float*)r->params.p;
  ad.g = (float*)r->grad.p;
  ad.m = (float*)r->m.p;
  ad.v = (float*)r->v.p;
  ad.packed = (uint8_t*)r->packed.p;
  ad.lr = r->cfg.lr;
  ad.b1 = r->cfg.beta1;
  ad.b2 = r->cfg.beta2;
  ad.eps = r->cfg.eps;
  ad.c1 = 1.f - powf(r->cfg.beta1, (float)r->step);
  ad.c2 = 1.f - powf(r->cfg.beta2, (float)r->step);
  ad.apply = 1;
  float* gp = (float*)r->gpart.p;
  void* args[] = {(void*)&r->nd, (void*)&recs, (void*)&pnv, (void*)&targets, (void*)&count, (void*)&cap,
                  (void*)&gp, (void*)&status, (void*)&ad};
  cudaError_t e = cudaLaunchCooperativeKernel((void*)k_nrc_train, r->sm_count, kTrainThreads, args, kTrainSmem, st);
  if (e != cudaSuccess) return cuda_error(e, "nrc train (cooperative launch)");
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
  r->infer_blocks = r->sm_count * 3;   // 64 KB of shared memory and 64 tensor-memory columns each: three an SM
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
  return nrc_infer_launch(r, nullptr, nullptr, (unsigned)n, nullptr, out_dev, s->status, (cudaStream_t)stream,
                          nullptr, pnv_dev);
}

// One training step on n given samples (p, n, v) with targets (n x 3):
// gradients (rt_nrc_get_grads), then Adam.
rt_status rt_nrc_train_step(rt_nrc* r, rt_scene* s, const float* pnv_dev, const float* target_dev, int64_t n,
                            void* stream) {
  if (!r || !s || n <= 0 || n > (1 << 26) || !pnv_dev || !target_dev)
    return set_error(RT_ERR_INVALID_ARG, "rt_nrc_train_step: bad argument");
  return nrc_train_launch(r, nullptr, target_dev, nullptr, (unsigned)n, s->status, (cudaStream_t)stream, pnv_dev);
}

}  // extern "C"
