// nrc_internal.cuh - shared declarations of the radiance-cache code.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rtb.h"

namespace rtb {

constexpr int kFeatures = 81;                          // encoded features (padded to 96)
constexpr int kNW = 64 * 96 + 3 * 64 * 64 + 3 * 64;    // weights, oracle layout
constexpr int kNB = 4 * 64 + 3;                        // biases
constexpr int kNP = kNW + kNB;                         // 18,883 parameters
constexpr unsigned kErrNrcTimeout = 8u;                // a tensor-core wait timed out

// What the cache kernels read, by value.
struct NrcDevice {
  const void* packed;     // BF16 forward weights (shared-memory image) then FP32 biases
  float* target;          // training targets of the current frame (3 per slot)
  float lo[3], inv_ext[3];
};

// Inference over `count` records, adding weight x radiance to fb (or, with
// fbs set, to fbs[frame] with the frame index in the record's last word).
// With pnv set, the first cap rows of pnv (n x 9) instead of records, weight 1, outputs to out3.
rt_status nrc_infer_launch(rt_nrc* r, const float4* recs, const unsigned* count, unsigned cap, float* fb, float* out3,
                           unsigned* status, cudaStream_t st, float* const* fbs = nullptr, const float* pnv = nullptr);
// Training on `count` (at most cap; all cap when count is null) stride-3
// records whose slot indexes targets, or, with pnv set, on the first cap
// rows of pnv (n x 9) and targets (n x 3); then the Adam step.
rt_status nrc_train_launch(rt_nrc* r, const float4* recs, const float* targets, const unsigned* count, unsigned cap,
                           unsigned* status, cudaStream_t st, const float* pnv = nullptr);
NrcDevice* nrc_device(rt_nrc* r);
const rt_scene* nrc_scene(const rt_nrc* r);   // the scene whose box normalises the encoding

// Per-frame buffers of a cached render.
struct NrcFrame {
  int depth;
  float* target;
  float4 *infer_q, *train_q;
  unsigned infer_cap, train_cap, train_batch;
  uint32_t seed;
};
rt_status nrc_frame_buffers(rt_nrc* r, int64_t ray_cap, bool train, NrcFrame* out);
// Cache hits of the previous frame (device), and the copy that keeps this frame's.
const unsigned* nrc_prev_hits(rt_nrc* r);
void nrc_keep_hits(rt_nrc* r, const unsigned* hits, cudaStream_t st);

}  // namespace rtb
