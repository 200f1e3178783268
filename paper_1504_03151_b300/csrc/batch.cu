// batch.cu - many scenes in one persistent launch (rt_batch_*).
//
// The paper renders one scene per run; a renderer that serves many scenes
// of uneven size and resolution wants them in one launch, so that small
// frames do not leave the GPU idle and large ones do not serialise the
// rest.  One kernel walks a global list of 32-pixel tiles of every frame
// (per-frame tile offsets, per-scene BVH and primitive pointers in a device
// table).  A warp takes a tile, traces its camera rays and then every ray
// they spawn - shadow rays to each point light (Alg. 1), reflection and
// refraction rays to max_depth (Sec. IV.A, Eq. 6-12) - depth first, with
// the extra rays of a hit shared among the warp's lanes through a pending
// stack in shared memory; then it takes the next tile, of any frame.  The
// launch (counter reset, image clears, kernel) is captured in a CUDA graph
// once per tune and replayed; an autotuner picks the tile shape, block size
// and grid size by timing them on the batch itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "nrc_internal.cuh"
#include "rtb_internal.cuh"
#include "trace_device.cuh"

namespace rtb {

// Pending rays a warp can share (48 B each; 6 KB a warp below 256-thread
// blocks, 3 KB in them, which keeps a block's static shared memory < 48 KB).
template <int kThreads>
__host__ __device__ constexpr int batch_pending() {
  return kThreads >= 256 ? 64 : 128;
}
// Blocks per SM the register budget is cut for (about 100 registers a thread).
template <int kThreads>
__host__ __device__ constexpr int batch_min_blocks() {
  return kThreads >= 256 ? 2 : 640 / kThreads;
}

struct BatchScene {
  DevScene sc;
  CamBasis cam;
  float* fb;
  int W, H, tiles_x;
  unsigned tile0;   // first tile of this frame in the global tile list
  int cap;          // traversal step cap
};

struct BatchCounts {
  unsigned rays[RT_MAX_DEPTH + 1];     // closest-hit rays traced at depth d
  unsigned shadow[RT_MAX_DEPTH + 1];   // shadow rays cast from depth-d hits
  unsigned hits[RT_MAX_DEPTH + 1];
  unsigned fetch;                      // next tile
  unsigned infer_count, train_count;   // radiance-cache records of the launch
  unsigned cache_hits;                 // hits at the cache depth
};

// The radiance cache in a batch (nrc_depth < 0: off): hits at nrc_depth
// push an inference record (p, pixel) (n) (-d) (w, frame) and end their
// path, except a seeded subset (probability train_batch / the previous
// launch's cache hits), which is traced on with unit weight into a training
// target (pixel ids < 0 route to target slot ~pixel).
struct BatchNrc {
  int depth;
  float4* infer_q;
  float4* train_q;
  float* target;
  unsigned infer_cap, train_cap, train_batch;
  const unsigned* prev_hits;
  uint32_t seed;
};

struct BatchParams {
  const BatchScene* scenes;
  int n;
  unsigned n_tiles;
  int max_depth;
  int tile_w, tile_h;
  float bg_r, bg_g, bg_b, eps_scale;
  BatchCounts* cnt;
  PassInfo ps;   // area-light samples and camera jitter: pass 0 of seed 0, no jitter
  BatchNrc nrc;
};

// Adds radiance to a pixel of the frame, or to a training target of the
// radiance cache when the path belongs to its training subset (pixel < 0).
__device__ __forceinline__ void add_rgb(float* fb, float* target, int pixel, f3 c) {
  float* p = pixel >= 0 ? fb + 3 * (size_t)pixel : target + 3 * (size_t)(~pixel);
  atomicAdd(p, c.x);
  atomicAdd(p + 1, c.y);
  atomicAdd(p + 2, c.z);
}

// kPass: some frame has area lights or emissive primitives (their sampling
// code is compiled only into these instances)
template <int kThreads, bool kPass>
__global__ void __launch_bounds__(kThreads, batch_min_blocks<kThreads>()) k_batch(BatchParams bp) {
  constexpr int kBatchPending = batch_pending<kThreads>();
  __shared__ int s_stack[kStackShared * kThreads];
  __shared__ float4 s_pend[kThreads / 32][kBatchPending][3];   // (o, pixel) (d, depth) (w, tmax)
  __shared__ int s_np[kThreads / 32];
  __shared__ unsigned s_cnt[3][RT_MAX_DEPTH + 1];
  int* stack = s_stack + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int i = threadIdx.x; i < 3 * (RT_MAX_DEPTH + 1); i += blockDim.x) (&s_cnt[0][0])[i] = 0u;
  if (lane == 0) s_np[warp] = 0;
  __syncthreads();
  const f3 bg = mk3(bp.bg_r, bp.bg_g, bp.bg_b);
  // second children this lane could not share (depth first: <= max_depth entries)
  float4 local[RT_MAX_DEPTH][3];
  int nl = 0;
  // A lane's item is a path segment (depth >= 0) or a shadow ray cast from a
  // depth-(~depth) hit (depth < 0; w is its contribution, tmax_item its length).
  bool have = false;
  f3 o = mk3(0, 0, 0), d = mk3(0, 0, 1), w = mk3(0, 0, 0);
  int depth = 0, pixel = 0;
  float tmax_item = 0.f;
  uint32_t code = 1u;   // path vertex of a segment's hit (keys the pass's samples)
  // the frame of the warp's current tile: every item of the warp belongs to it
  DevScene sc;
  sc.n_prims = 0;
  float* fb = nullptr;
  float* const target = bp.nrc.target;
  int cap = 0, frame = 0;
  WorkCount wc = {0u, 0u, 0u, 0u};
  for (;;) {
    // --- refill lanes without an item: own overflow, then the warp's stack
    if (!have && nl > 0) {
      --nl;
      o = xyz(local[nl][0]);
      pixel = __float_as_int(local[nl][0].w);
      d = xyz(local[nl][1]);
      depth = __float_as_int(local[nl][1].w);
      w = xyz(local[nl][2]);
      code = __float_as_uint(local[nl][2].w);
      have = true;
    }
    __syncwarp();   // rays pushed by this warp's lanes are visible
    unsigned need = __ballot_sync(kFull, !have);
    int np = s_np[warp];
    if (need && np > 0) {
      int take = min(__popc(need), np);
      int rank = __popc(need & lt);
      if (!have && rank < take) {
        const float4* r = s_pend[warp][np - 1 - rank];
        o = xyz(r[0]);
        pixel = __float_as_int(r[0].w);
        d = xyz(r[1]);
        depth = __float_as_int(r[1].w);
        w = xyz(r[2]);
        tmax_item = r[2].w;              // a shadow ray's length,
        code = __float_as_uint(r[2].w);  // or a segment's path vertex
        have = true;
      }
      __syncwarp();
      if (lane == 0) s_np[warp] = np - take;
      __syncwarp();
    }
    if (!__any_sync(kFull, have)) {
      // --- the warp is idle (no item, nothing pending): the next tile
      unsigned t = 0;
      if (lane == 0) t = atomicAdd(&bp.cnt->fetch, 1u);
      t = __shfl_sync(kFull, t, 0);
      if (t >= bp.n_tiles) break;
      int lo = 0, hi = bp.n - 1;   // the frame whose tiles start last at or before t
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&bp.scenes[mid].tile0) <= t) lo = mid;
        else hi = mid - 1;
      }
      const BatchScene* bs = bp.scenes + lo;
      frame = lo;
      sc = bs->sc;
      fb = bs->fb;
      cap = bs->cap;
      const int W = bs->W, H = bs->H;
      const unsigned k = t - bs->tile0;
      const int x = (int)(k % (unsigned)bs->tiles_x) * bp.tile_w + lane % bp.tile_w;
      const int y = (int)(k / (unsigned)bs->tiles_x) * bp.tile_h + lane / bp.tile_w;
      if (x < W && y < H) {
        const CamBasis cb = bs->cam;
        pixel = y * W + x;
        camera_ray(cb, W, H, x, y, o, d);   // pixel centres (the batch renders pass 0 without jitter)
        w = mk3(1.f, 1.f, 1.f);
        depth = 0;
        code = 1u;
        have = true;
      }
      continue;   // to the top: a tile cut by the image edge still has lanes with work
    }
    // --- one item per lane
    Children ch;
    ch.want_r = ch.want_t = ch.bounce = false;
    if (have && depth < 0) {
      bool sfail = false;
      float tm = tmax_item;
      int h = traverse<true, false, kThreads>(sc, make_ray(o, d), 0.0f, tm, stack, cap, sfail, wc);
      if (sfail) atomicOr(sc.status, kErrTraversalLimit);
      if (h < 0 && !sfail) add_rgb(fb, target, pixel, w);
    } else if (have) {
      float t = INFINITY;
      bool fail = false;
      int hit = traverse<false, false, kThreads>(sc, make_ray(o, d), 0.0f, t, stack, cap, fail, wc);
      if (fail) atomicOr(sc.status, kErrTraversalLimit);
      atomicAdd(&s_cnt[0][depth], 1u);
      bool live = hit >= 0;
      Surface sf;
      if (!live) {
        add_rgb(fb, target, pixel, w * bg);
      } else {
        atomicAdd(&s_cnt[2][depth], 1u);
        sf = surface_at(sc, hit, o, d, t, bp.eps_scale);
        // L_e (not on a diffuse bounce: its parent sampled the emitters)
        const bool via_bounce = kPass && (code & kCodeBounce) != 0u;
        if (!via_bounce && (sf.emission.x != 0.f || sf.emission.y != 0.f || sf.emission.z != 0.f))
          add_rgb(fb, target, pixel, w * sf.emission);
        if (depth == bp.nrc.depth) {
          // the radiance cache: this hit's radiance comes from the network
          atomicAdd(&bp.cnt->cache_hits, 1u);
          const unsigned pos = atomicAdd(&bp.cnt->infer_count, 1u);
          if (pos < bp.nrc.infer_cap) {
            float4* q = bp.nrc.infer_q + 4 * (size_t)pos;
            q[0] = make_float4(sf.p.x, sf.p.y, sf.p.z, __int_as_float(pixel));
            q[1] = make_float4(sf.n.x, sf.n.y, sf.n.z, 0.f);
            q[2] = make_float4(-d.x, -d.y, -d.z, 0.f);
            q[3] = make_float4(w.x, w.y, w.z, __int_as_float(frame));
          } else {
            atomicOr(sc.status, kErrQueueOverflow);
          }
          const unsigned prev = bp.nrc.prev_hits ? *bp.nrc.prev_hits : 0u;
          const float u = (float)(hash32(bp.nrc.seed ^ hash32((uint32_t)pixel * 0x9E3779B9u ^
                                                               __float_as_uint(d.x) ^ (uint32_t)frame * 0x85EBCA6Bu)) >>
                                  8) *
                          (1.0f / 16777216.0f);
          const bool sel = bp.nrc.train_batch > 0 && (prev == 0u || (float)bp.nrc.train_batch > u * (float)prev);
          const unsigned slot = sel ? atomicAdd(&bp.cnt->train_count, 1u) : 0u;
          if (sel && slot < bp.nrc.train_cap) {
            float4* q = bp.nrc.train_q + 3 * (size_t)slot;
            q[0] = make_float4(sf.p.x, sf.p.y, sf.p.z, __int_as_float((int)slot));
            q[1] = make_float4(sf.n.x, sf.n.y, sf.n.z, 0.f);
            q[2] = make_float4(-d.x, -d.y, -d.z, 0.f);
            w = mk3(1.f, 1.f, 1.f);
            pixel = ~(int)slot;   // traced on, with unit weight, into the training target
          } else {
            live = false;          // this path ends in the cache
          }
        }
      }
      if (live) {
        const uint32_t vcode = kPass ? (code & ~kCodeBounce) : code;
        if (sf.kind != RT_MAT_DIELECTRIC && (1.f - sf.rho) > 0.f) {
          // point lights, then one sampled point of each area light and emitter
          for (int li = 0; li < sc.n_lights + (kPass ? sc.n_alights + sc.n_emitters : 0); ++li) {
            f3 contrib, os, sd;
            float tmax;
            bool lit;
            if (li < sc.n_lights) {
              lit = light_term(sf, d, w, __ldg(&sc.lights[2 * li]), __ldg(&sc.lights[2 * li + 1]), contrib, os, sd,
                               tmax);
            } else {
              lit = false;
              if constexpr (kPass) {
                float a, b;
                pass_sample(bp.ps, pixel, vcode, (uint32_t)(li - sc.n_lights), a, b);
                lit = area_term(sf, d, w, area_point(sc, li - sc.n_lights, a, b), contrib, os, sd, tmax);
              }
            }
            if (!lit) continue;
            atomicAdd(&s_cnt[1][depth], 1u);
            // to the warp's pending stack for a free lane; traced here when it is full
            int pos = atomicAdd(&s_np[warp], 1);
            if (pos < kBatchPending) {
              float4* r = s_pend[warp][pos];
              r[0] = make_float4(os.x, os.y, os.z, __int_as_float(pixel));
              r[1] = make_float4(sd.x, sd.y, sd.z, __int_as_float(~depth));
              r[2] = make_float4(contrib.x, contrib.y, contrib.z, tmax);
              continue;
            }
            atomicSub(&s_np[warp], 1);
            bool sfail = false;
            int h = traverse<true, false, kThreads>(sc, make_ray(os, sd), 0.0f, tmax, stack, cap, sfail, wc);
            if (sfail) atomicOr(sc.status, kErrTraversalLimit);
            if (h < 0 && !sfail) add_rgb(fb, target, pixel, contrib);
          }
        }
        if (depth < bp.max_depth) {
          ch = children_of(sf, d, w);
          if (kPass && bp.ps.bounce) add_bounce(ch, sf, w, bp.ps, pixel, vcode);
        }
      }
    }
    // --- a second child goes to the warp's stack (or this lane's overflow)
    bool two = have && ch.want_r && ch.want_t;
    unsigned m2 = __ballot_sync(kFull, two);
    if (m2) {
      __syncwarp();
      int np2 = s_np[warp];
      int room = kBatchPending - np2;
      int rank = __popc(m2 & lt);
      float4 r0 = make_float4(ch.or_.x, ch.or_.y, ch.or_.z, __int_as_float(pixel));
      float4 r1 = make_float4(ch.dr.x, ch.dr.y, ch.dr.z, __int_as_float(depth + 1));
      float4 r2 = make_float4(ch.wr.x, ch.wr.y, ch.wr.z, __uint_as_float(code << 1));
      if (two) {
        if (rank < room) {
          float4* r = s_pend[warp][np2 + rank];
          r[0] = r0;
          r[1] = r1;
          r[2] = r2;
        } else if (nl < RT_MAX_DEPTH) {
          local[nl][0] = r0;
          local[nl][1] = r1;
          local[nl][2] = r2;
          ++nl;
        } else {
          atomicOr(sc.status, kErrQueueOverflow);   // not reachable for depth <= 16
        }
      }
      __syncwarp();
      if (lane == 0) s_np[warp] = np2 + min(__popc(m2), room);
      __syncwarp();
    }
    // --- this lane follows its (other) child, or is free for new work
    if (have) {
      if (ch.want_t) {
        o = ch.ot;
        d = ch.dt;
        w = ch.wt;
        code = (code << 1) | 1u | (ch.bounce ? kCodeBounce : 0u);
        ++depth;
      } else if (ch.want_r) {
        o = ch.or_;
        d = ch.dr;
        w = ch.wr;
        code <<= 1;
        ++depth;
      } else {
        have = false;
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= RT_MAX_DEPTH; i += blockDim.x) {
    if (s_cnt[0][i]) atomicAdd(&bp.cnt->rays[i], s_cnt[0][i]);
    if (s_cnt[1][i]) atomicAdd(&bp.cnt->shadow[i], s_cnt[1][i]);
    if (s_cnt[2][i]) atomicAdd(&bp.cnt->hits[i], s_cnt[2][i]);
  }
}

using BatchKernel = void (*)(BatchParams);

static BatchKernel batch_kernel(int threads, bool pass = false) {
  switch (threads) {
    case 64:
      return pass ? k_batch<64, true> : k_batch<64, false>;
    case 128:
      return pass ? k_batch<128, true> : k_batch<128, false>;
    case 256:
      return pass ? k_batch<256, true> : k_batch<256, false>;
    default:
      return nullptr;
  }
}

static bool valid_tune(const rt_tune& t) {
  return t.tile_w > 0 && t.tile_h > 0 && t.tile_w * t.tile_h == 32 && batch_kernel(t.block_threads) &&
         t.blocks_per_sm >= 0;
}

static bool same_tune(const rt_tune& a, const rt_tune& b) {
  return a.tile_w == b.tile_w && a.tile_h == b.tile_h && a.block_threads == b.block_threads &&
         a.blocks_per_sm == b.blocks_per_sm;
}

static rt_tune default_tune() {
  rt_tune t;
  t.tile_w = 8;
  t.tile_h = 4;
  t.block_threads = 128;
  t.blocks_per_sm = 0;
  return t;
}

}  // namespace rtb

using namespace rtb;

struct rt_batch {
  std::vector<rt_scene*> scenes;
  std::vector<rt_camera> cams;
  std::vector<int> W, H;
  std::vector<float*> outs;
  int n = 0, max_depth = 0;
  rt_render_options opt;
  int device = 0, sm_count = 0;
  Buf table, counts;
  Buf fbs;                            // device array of the frames' images (the cache's inference adds there)
  BatchScene* host_table = nullptr;   // pinned staging of the device table
  cudaStream_t cap_stream = nullptr;  // graphs are captured here (never the caller's stream)
  struct Graph {
    rt_tune tune;
    bool pass;   // the kernel with area-light sampling
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  rt_tune best;
  bool tuned = false;
};

namespace rtb {

// Fills the device table for `tune` (through the pinned staging copy) and
// returns the number of tiles; the copy is ordered on `st`.
static rt_status batch_table(rt_batch* b, const rt_tune& tune, unsigned* n_tiles, cudaStream_t st) {
  uint64_t tile0 = 0;
  for (int i = 0; i < b->n; ++i) {
    rt_scene* s = b->scenes[i];
    if (!s->built) return set_error(RT_ERR_NOT_BUILT, "rt_batch_render: a scene of the batch has no BVH");
    BatchScene& e = b->host_table[i];
    e.sc = dev_scene(s, true);
    e.cam = camera_basis(&b->cams[i], b->W[i], b->H[i]);
    e.fb = b->outs[i];
    e.W = b->W[i];
    e.H = b->H[i];
    e.tiles_x = (e.W + tune.tile_w - 1) / tune.tile_w;
    const int tiles_y = (e.H + tune.tile_h - 1) / tune.tile_h;
    e.tile0 = (unsigned)tile0;
    int64_t tcap = b->opt.traversal_cap > 0 ? b->opt.traversal_cap : 4 * std::max<int64_t>(s->n_nodes4, 1) + 64;
    e.cap = (int)std::min<int64_t>(tcap, 0x7fffffff);
    tile0 += (uint64_t)e.tiles_x * tiles_y;
  }
  if (tile0 > 0xffffffffull) return set_error(RT_ERR_UNSUPPORTED, "rt_batch_render: more than 2^32 tiles");
  *n_tiles = (unsigned)tile0;
  return cuda_error(cudaMemcpyAsync(b->table.p, b->host_table, sizeof(BatchScene) * b->n, cudaMemcpyHostToDevice, st),
                    "rt_batch_render: table");
}

// Blocks of the persistent grid for a tune: as many as fit, or the tune's cap a SM.
static rt_status batch_grid(const rt_batch* b, const rt_tune& tune, BatchKernel kern, int* grid) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tune.block_threads, 0);
  if (e != cudaSuccess) return cuda_error(e, "rt_batch_render: occupancy");
  if (per_sm < 1) return set_error(RT_ERR_UNSUPPORTED, "rt_batch_render: the kernel does not fit on an SM");
  if (tune.blocks_per_sm > 0) per_sm = std::min(per_sm, tune.blocks_per_sm);
  *grid = b->sm_count * per_sm;
  return RT_OK;
}

// The kernel's parameters for a tune, with the radiance cache off.
static BatchParams batch_params(const rt_batch* b, const rt_tune& tune, unsigned n_tiles) {
  BatchParams bp;
  bp.scenes = (const BatchScene*)b->table.p;
  bp.n = b->n;
  bp.n_tiles = n_tiles;
  bp.max_depth = b->max_depth;
  bp.tile_w = tune.tile_w;
  bp.tile_h = tune.tile_h;
  bp.bg_r = b->opt.background[0];
  bp.bg_g = b->opt.background[1];
  bp.bg_b = b->opt.background[2];
  bp.eps_scale = b->opt.eps_scale;
  bp.cnt = (BatchCounts*)b->counts.p;
  memset(&bp.ps, 0, sizeof(bp.ps));
  bp.ps.strata = 1;
  bp.ps.bounce = (b->opt.flags & RT_FLAG_DIFFUSE_BOUNCE) != 0;
  memset(&bp.nrc, 0, sizeof(bp.nrc));
  bp.nrc.depth = -1;
  return bp;
}

// Whether the batch needs the kernel instance with the sampling code.
static bool batch_pass(const rt_batch* b) {
  bool pass = (b->opt.flags & RT_FLAG_DIFFUSE_BOUNCE) != 0;
  for (rt_scene* s : b->scenes) pass = pass || s->n_alights > 0 || s->n_emitters > 0;
  return pass;
}

// The launch of one tune: counters, image clears and the kernel, captured
// on the batch's own stream into a graph (once per tune).
static rt_status batch_graph(rt_batch* b, const rt_tune& tune, bool pass, unsigned n_tiles, cudaGraphExec_t* exec) {
  for (auto& g : b->graphs)
    if (same_tune(g.tune, tune) && g.pass == pass) {
      *exec = g.exec;
      return RT_OK;
    }
  BatchKernel kern = batch_kernel(tune.block_threads, pass);
  int grid = 0;
  rt_status rs = batch_grid(b, tune, kern, &grid);
  if (rs) return rs;
  BatchParams bp = batch_params(b, tune, n_tiles);
  cudaError_t e;
  cudaStream_t cs = b->cap_stream;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_error(e, "rt_batch_render: begin capture");
  cudaMemsetAsync(b->counts.p, 0, sizeof(BatchCounts), cs);
  for (int i = 0; i < b->n; ++i) cudaMemsetAsync(b->outs[i], 0, (size_t)b->W[i] * b->H[i] * 3 * sizeof(float), cs);
  kern<<<grid, tune.block_threads, 0, cs>>>(bp);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  e = cudaGetLastError();
  if (e2 != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_error(e2 != cudaSuccess ? e2 : e, "rt_batch_render: capture");
  }
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_error(e, "rt_batch_render: instantiate");
  b->graphs.push_back({tune, pass, x});
  *exec = x;
  return RT_OK;
}

static rt_status batch_render(rt_batch* b, const rt_tune& tune, cudaStream_t st) {
  if (!valid_tune(tune))
    return set_error(RT_ERR_INVALID_ARG, "rt_batch_render: tune needs tile_w * tile_h == 32, block_threads 64, "
                                         "128 or 256 and blocks_per_sm >= 0");
  unsigned n_tiles = 0;
  rt_status rs = batch_table(b, tune, &n_tiles, st);
  if (rs) return rs;
  const bool pass = batch_pass(b);
  cudaGraphExec_t exec = nullptr;
  if ((rs = batch_graph(b, tune, pass, n_tiles, &exec))) return rs;
  // the tile count depends only on the sizes and the tile shape, both fixed per graph
  return cuda_error(cudaGraphLaunch(exec, st), "rt_batch_render: launch");
}

}  // namespace rtb

extern "C" {

rt_status rt_batch_create(rt_scene* const* scenes, int32_t n, const rt_camera* cameras, const int32_t* widths,
                          const int32_t* heights, int32_t max_depth, float* const* out_rgb,
                          const rt_render_options* options, rt_batch** out) {
  if (!scenes || !cameras || !widths || !heights || !out_rgb || !out)
    return set_error(RT_ERR_INVALID_ARG, "rt_batch_create: NULL argument");
  *out = nullptr;
  if (n < 1) return set_error(RT_ERR_INVALID_ARG, "rt_batch_create: n < 1");
  if (max_depth < 0 || max_depth > RT_MAX_DEPTH)
    return set_error(RT_ERR_INVALID_ARG, "rt_batch_create: max_depth outside [0, 16]");
  rt_render_options opt;
  rt_render_options_default(&opt);
  if (options) opt = *options;
  if (!opt.use_bvh) return set_error(RT_ERR_INVALID_ARG, "rt_batch_create: batches trace with the BVH (use_bvh)");
  if (opt.flags & RT_FLAG_DETERMINISTIC)
    return set_error(RT_ERR_UNSUPPORTED, "rt_batch_create: a batch does not take RT_FLAG_DETERMINISTIC");
  if (!std::isfinite(opt.background[0]) || !std::isfinite(opt.background[1]) || !std::isfinite(opt.background[2]) ||
      !std::isfinite(opt.eps_scale) || opt.eps_scale < 0.f || opt.traversal_cap < 0)
    return set_error(RT_ERR_INVALID_ARG, "rt_batch_create: invalid options");
  for (int i = 0; i < n; ++i) {
    if (!scenes[i] || !out_rgb[i]) return set_error(RT_ERR_INVALID_ARG, "rt_batch_create: NULL scene or image");
    if (widths[i] < 1 || heights[i] < 1) return set_error(RT_ERR_INVALID_ARG, "rt_batch_create: size < 1");
    if ((int64_t)widths[i] * heights[i] > (int64_t)1 << 30)
      return set_error(RT_ERR_UNSUPPORTED, "rt_batch_create: image too large");
    if (!finite_cam(&cameras[i])) return set_error(RT_ERR_INVALID_ARG, "rt_batch_create: invalid camera");
    if (scenes[i]->device != scenes[0]->device)
      return set_error(RT_ERR_INVALID_ARG, "rt_batch_create: scenes on different devices");
  }
  rt_batch* b = new rt_batch();
  b->scenes.assign(scenes, scenes + n);
  b->cams.assign(cameras, cameras + n);
  b->W.assign(widths, widths + n);
  b->H.assign(heights, heights + n);
  b->outs.assign(out_rgb, out_rgb + n);
  b->n = n;
  b->max_depth = max_depth;
  b->opt = opt;
  b->device = scenes[0]->device;
  b->sm_count = scenes[0]->sm_count;
  b->best = default_tune();
  rt_status rs = RT_OK;
  cudaError_t e = cudaSetDevice(b->device);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->host_table, sizeof(BatchScene) * n);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) rs = cuda_error(e, "rt_batch_create");
  if (!rs) rs = ensure(b->table, sizeof(BatchScene) * n);
  if (!rs) rs = ensure(b->counts, sizeof(BatchCounts));
  if (rs) {
    rt_batch_destroy(b);
    return rs;
  }
  *out = b;
  return RT_OK;
}

rt_status rt_batch_set_cameras(rt_batch* b, const rt_camera* cameras) {
  if (!b || !cameras) return set_error(RT_ERR_INVALID_ARG, "rt_batch_set_cameras: NULL argument");
  for (int i = 0; i < b->n; ++i)
    if (!finite_cam(&cameras[i])) return set_error(RT_ERR_INVALID_ARG, "rt_batch_set_cameras: invalid camera");
  b->cams.assign(cameras, cameras + b->n);
  return RT_OK;
}

}  // extern "C"

namespace rtb {

// Sums the launch's counters into *stats (syncs `stream`) and returns the
// scenes' latched errors.
static rt_status batch_stats(rt_batch* b, rt_render_stats* stats, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "rt_batch_render");
  BatchCounts c;
  e = cudaMemcpy(&c, b->counts.p, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "rt_batch_render: stats");
  memset(stats, 0, sizeof(*stats));
  for (int d = 0; d <= RT_MAX_DEPTH; ++d) {
    stats->rays_per_depth[d] = c.rays[d];
    stats->shadow_per_depth[d] = c.shadow[d];
    stats->hits_per_depth[d] = c.hits[d];
    stats->shadow += c.shadow[d];
    if (d == 0) stats->primary = c.rays[0];
    else stats->secondary += c.rays[d];
  }
  for (int i = 0; i < b->n; ++i) {
    rt_status rs = rt_scene_sync(b->scenes[i], stream);
    if (rs) return rs;
  }
  return RT_OK;
}

}  // namespace rtb

extern "C" {

rt_status rt_batch_render(rt_batch* b, const rt_tune* tune, rt_render_stats* stats, void* stream) {
  if (!b) return set_error(RT_ERR_INVALID_ARG, "rt_batch_render: batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  // the staging copy of the previous render may still be in flight
  cudaError_t e = cudaStreamSynchronize(b->cap_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "rt_batch_render");
  rt_status rs = batch_render(b, tune ? *tune : b->best, st);
  if (rs) return rs;
  if (!stats) return RT_OK;
  rs = batch_stats(b, stats, stream);
  if (!rs) stats->launches = 1;
  return rs;
}

rt_status rt_batch_render_nrc(rt_batch* b, rt_nrc* nrc, int train, const rt_tune* tune_in, rt_render_stats* stats,
                              void* stream) {
  if (!b || !nrc) return set_error(RT_ERR_INVALID_ARG, "rt_batch_render_nrc: NULL batch or cache");
  for (int i = 0; i < b->n; ++i)
    if (b->scenes[i] != nrc_scene(nrc))
      return set_error(RT_ERR_INVALID_ARG, "rt_batch_render_nrc: every frame must show the scene of the cache");
  if (b->opt.flags & RT_FLAG_DIFFUSE_BOUNCE)
    return set_error(RT_ERR_UNSUPPORTED, "rt_batch_render_nrc: the radiance cache does not take RT_FLAG_DIFFUSE_BOUNCE");
  const rt_tune tune = tune_in ? *tune_in : b->best;
  if (!valid_tune(tune))
    return set_error(RT_ERR_INVALID_ARG, "rt_batch_render_nrc: tune needs tile_w * tile_h == 32, block_threads 64, "
                                         "128 or 256 and blocks_per_sm >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(b->cap_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "rt_batch_render_nrc");
  unsigned n_tiles = 0;
  rt_status rs = batch_table(b, tune, &n_tiles, st);
  if (rs) return rs;
  // inference records: up to two children per dielectric hit above the cache
  // depth; 2 x the batch's pixels is the frames' ray-queue default
  int64_t pixels = 0;
  for (int i = 0; i < b->n; ++i) pixels += (int64_t)b->W[i] * b->H[i];
  NrcFrame nf;
  if ((rs = nrc_frame_buffers(nrc, std::min<int64_t>(2 * pixels, 0x7fffffff), train != 0, &nf))) return rs;
  if (!b->fbs.p) {
    if ((rs = ensure(b->fbs, sizeof(float*) * b->n))) return rs;
    e = cudaMemcpy(b->fbs.p, b->outs.data(), sizeof(float*) * b->n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "rt_batch_render_nrc: image table");
  }
  const bool pass = batch_pass(b);
  BatchKernel kern = batch_kernel(tune.block_threads, pass);
  int grid = 0;
  if ((rs = batch_grid(b, tune, kern, &grid))) return rs;
  BatchParams bp = batch_params(b, tune, n_tiles);
  const int T = nf.depth <= b->max_depth ? nf.depth : -1;
  bp.nrc.depth = T;
  bp.nrc.infer_q = nf.infer_q;
  bp.nrc.train_q = nf.train_q;
  bp.nrc.target = nf.target;
  bp.nrc.infer_cap = nf.infer_cap;
  bp.nrc.train_cap = nf.train_cap;
  bp.nrc.train_batch = train ? nf.train_batch : 0u;
  bp.nrc.prev_hits = nrc_prev_hits(nrc);
  bp.nrc.seed = nf.seed;
  BatchCounts* cnt = (BatchCounts*)b->counts.p;
  unsigned* status = b->scenes[0]->status;
  if (T >= 0 && train) cudaMemsetAsync(nf.target, 0, (size_t)nf.train_cap * 12, st);
  cudaMemsetAsync(cnt, 0, sizeof(BatchCounts), st);
  for (int i = 0; i < b->n; ++i) cudaMemsetAsync(b->outs[i], 0, (size_t)b->W[i] * b->H[i] * 3 * sizeof(float), st);
  kern<<<grid, tune.block_threads, 0, st>>>(bp);
  int launches = 1;
  if (T >= 0) {
    // the cache's answers for every frame's hits at depth T, then one
    // training step on the launch's targets
    if ((rs = nrc_infer_launch(nrc, nf.infer_q, &cnt->infer_count, nf.infer_cap, nullptr, nullptr, status, st,
                               (float* const*)b->fbs.p)))
      return rs;
    nrc_keep_hits(nrc, &cnt->cache_hits, st);
    launches += 1;
    if (train) {
      if ((rs = nrc_train_launch(nrc, nf.train_q, nf.target, &cnt->train_count, nf.train_cap, status, st))) return rs;
      launches += 3;
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "rt_batch_render_nrc: launch");
  if (!stats) return RT_OK;
  rs = batch_stats(b, stats, stream);
  if (!rs) stats->launches = launches;
  return rs;
}

rt_status rt_batch_autotune(rt_batch* b, rt_tune* best, float* best_ms, void* stream) {
  if (!b) return set_error(RT_ERR_INVALID_ARG, "rt_batch_autotune: batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const int tiles[4][2] = {{8, 4}, {4, 8}, {16, 2}, {32, 1}};
  const int threads[3] = {64, 128, 256};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_error(e, "rt_batch_autotune");
  rt_status rs = RT_OK;
  float best_t = INFINITY;
  rt_tune choice = default_tune();
  for (int ti = 0; ti < 4 && !rs; ++ti) {
    for (int bi = 0; bi < 3 && !rs; ++bi) {
      rt_tune t;
      t.tile_w = tiles[ti][0];
      t.tile_h = tiles[ti][1];
      t.block_threads = threads[bi];
      t.blocks_per_sm = 0;
      float ms = 0.f;
      for (int rep = 0; rep < 3 && !rs; ++rep) {   // the first is a warm-up (and the graph's capture)
        e = cudaStreamSynchronize(b->cap_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
          rs = cuda_error(e, "rt_batch_autotune");
          break;
        }
        cudaEventRecord(e0, st);
        rs = batch_render(b, t, st);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (!rs && e != cudaSuccess) rs = cuda_error(e, "rt_batch_autotune");
        float x = 0.f;
        if (!rs) cudaEventElapsedTime(&x, e0, e1);
        if (rep > 0) ms += x;
      }
      if (!rs && ms / 2 < best_t) {
        best_t = ms / 2;
        choice = t;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rs) return rs;
  b->best = choice;
  b->tuned = true;
  if (best) *best = choice;
  if (best_ms) *best_ms = best_t;
  // the images of the chosen tune
  rs = batch_render(b, choice, st);
  if (rs) return rs;
  for (int i = 0; i < b->n; ++i) {
    rs = rt_scene_sync(b->scenes[i], stream);
    if (rs) return rs;
  }
  return RT_OK;
}

rt_status rt_render_batch(rt_scene* const* scenes, const rt_camera* cameras, const int32_t* widths,
                          const int32_t* heights, int32_t n, int32_t max_depth, float* const* out_rgb,
                          const rt_tune* tune, void* stream) {
  rt_batch* b = nullptr;
  rt_status rs = rt_batch_create(scenes, n, cameras, widths, heights, max_depth, out_rgb, nullptr, &b);
  if (rs) return rs;
  rs = rt_batch_render(b, tune, nullptr, stream);
  // the batch's tables must outlive its launch
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (!rs && e != cudaSuccess) rs = cuda_error(e, "rt_render_batch");
  for (int i = 0; !rs && i < n; ++i) rs = rt_scene_sync(scenes[i], stream);
  rt_batch_destroy(b);
  return rs;
}

rt_status rt_batch_destroy(rt_batch* b) {
  if (!b) return RT_OK;
  if (b->cap_stream) cudaStreamSynchronize(b->cap_stream);
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  release(b->table);
  release(b->counts);
  release(b->fbs);
  if (b->host_table) cudaFreeHost(b->host_table);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
  return RT_OK;
}

}  // extern "C"
