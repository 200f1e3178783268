// bvh.cu - on-device BVH build: Morton codes, radix sort, LBVH hierarchy,
// bottom-up boxes with SAH costs, binned-SAH rebuild of the top levels over
// Morton clusters, SAH leaf collapsing, traversal layout.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <utility>
#include <vector>

#include "rtb_internal.cuh"

namespace cg = cooperative_groups;

namespace rtb {

constexpr int kSortTile = 4096;     // keys per radix-sort tile (256 threads x 16)
constexpr int kScanBlock = 4096;    // elements per scan block (1024 threads x 4)
constexpr int kSortCoopMaxBlocks = 1024;   // grid of the single-launch sort (co-resident blocks)
constexpr int kSortCoopMaxKeys = 1 << 22;  // larger inputs take the multi-launch sort
constexpr int kTopBins = 16;        // SAH bins per axis for the top-level rebuild
constexpr int kTopMaxLevels = 64;   // launches of the level kernel (empty ones return at once)
constexpr int kTopCache = 4096;     // clusters of one segment held in shared memory (41 B each)
// A segment of more clusters bins an even subsample of about this many to
// choose its split plane (the partition still takes every cluster).  On the
// 1080p terrain the root's 3,299 clusters bin every 7th (472), the next
// levels' 1,650 and 825 every 4th and every 2nd (413 each): the build is
// 6 us shorter than with a subsample of 1024, and the tree's SAH cost 28.48
// against 28.50 (with 256: 28.61).
constexpr int kTopSample = 512;
constexpr int kTopWarpSeg = 32;     // segments of at most this many clusters are finished by one warp
constexpr int kTopForceMedian = 32; // from this level on, split segments at the middle: with at
                                    // most 2^28 clusters every segment is done by level 60

// Device-side build results, read by rt_bvh_get_info.
struct BuildInfo {
  int height;          // deepest internal-node chain (stack entries needed <= height)
  float sah;           // SAH cost of the final tree
  float sah_lbvh;      // SAH cost of the plain LBVH (single-primitive leaves)
  int n_clusters;
  int n_top;           // top nodes emitted by the SAH rebuild
  int root;
  int max_leaf;
  int pad;
};

// Scratch carved out of one allocation.
struct BuildScratch {
  float4 *aabb_lo, *aabb_hi;     // per primitive (id order)
  unsigned *keys0, *vals0, *keys1, *vals1;
  unsigned* hist;                // 256 x tiles
  unsigned* partials;            // scan partials
  int *lch, *rch, *parent, *leaf_parent, *flags;
  int2* range;
  float4 *node_lo, *node_hi;     // LBVH internal boxes; lo.w = SAH cost, hi.w = meta bits
  float* cost_lbvh;
  int* cent_bounds;              // 6 ordered ints
  // top-level rebuild
  // The cluster list, in two ping-pong buffers (a, b) that hold per
  // position a cluster's id and its box (lo.w = primitive count, hi.w =
  // height).  k_find_clusters fills buffer a with id = position.
  int *clu_a, *clu_b;
  int* clu_link;                 // per cluster id: its link (internal LBVH node or leaf link)
  float4 *clu_lo, *clu_hi;       // buffer a's boxes
  float4 *clu_lo_b, *clu_hi_b;   // buffer b's boxes
  int4 *seg_a, *seg_b;           // active segments: (begin, end, parent slot, node id)
  int* seg_count;                // [level] segments; [kTopMaxLevels + 1] clusters; [kTopMaxLevels + 2] small segments
  int* top_count;
  int4* small_seg;               // segments of <= kTopWarpSeg clusters: (begin, end, top node, level)
  BuildInfo* info;
};

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// One buffer of the top rebuild's cluster list: a split reads a segment's
// ids and boxes by position, all in one round trip, and writes them in
// their new order to the other buffer.
struct CluList {
  int* id;
  float4* lo;
  float4* hi;
};

// ---------------------------------------------------------------------------
// ordered-int encoding of floats for atomic min / max
// ---------------------------------------------------------------------------
__device__ __forceinline__ int f2o(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__device__ __forceinline__ float area(float4 lo, float4 hi) {
  float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
  if (!(dx >= 0.f) || !(dy >= 0.f) || !(dz >= 0.f)) return 0.f;
  return 2.f * (dx * dy + dy * dz + dz * dx);
}

// Grows a box by a few ulps so that the slab test never cuts off a
// primitive that lies on its face.
__device__ __forceinline__ float pad_lo(float x) { return x - fabsf(x) * 2.4e-7f - 1e-30f; }
__device__ __forceinline__ float pad_hi(float x) { return x + fabsf(x) * 2.4e-7f + 1e-30f; }

// ---------------------------------------------------------------------------
// 1. primitive boxes and the centroid bounds
// ---------------------------------------------------------------------------
// The centroid bounds' reset value (an empty box).  The kernel that follows
// the last reader of the bounds in a build (k_hierarchy, or k_layout_single)
// resets them for the next build; k_init_bounds runs only on fresh scratch.
__device__ __forceinline__ void reset_bounds(int* cb, int t) {
  if (t < 3) cb[t] = f2o(INFINITY);
  else if (t < 6) cb[t] = f2o(-INFINITY);
}
__global__ void k_init_bounds(int* cb) { reset_bounds(cb, threadIdx.x); }

__global__ void k_prim_bounds(const float4* __restrict__ prims, int n, float4* __restrict__ lo_out,
                              float4* __restrict__ hi_out, int* __restrict__ cb) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  float cx = INFINITY, cy = INFINITY, cz = INFINITY, Cx = -INFINITY, Cy = -INFINITY, Cz = -INFINITY;
  if (i < n) {
    float4 r0 = prims[3 * (size_t)i], r1 = prims[3 * (size_t)i + 1], r2 = prims[3 * (size_t)i + 2];
    float4 lo, hi;
    if (__float_as_int(r0.w) == kKindSphere) {
      float r = r1.x;
      lo = make_float4(r0.x - r, r0.y - r, r0.z - r, 0.f);
      hi = make_float4(r0.x + r, r0.y + r, r0.z + r, 0.f);
    } else {
      float ax = r0.x + r1.x, ay = r0.y + r1.y, az = r0.z + r1.z;
      float bx = r0.x + r2.x, by = r0.y + r2.y, bz = r0.z + r2.z;
      lo = make_float4(fminf(r0.x, fminf(ax, bx)), fminf(r0.y, fminf(ay, by)), fminf(r0.z, fminf(az, bz)), 0.f);
      hi = make_float4(fmaxf(r0.x, fmaxf(ax, bx)), fmaxf(r0.y, fmaxf(ay, by)), fmaxf(r0.z, fmaxf(az, bz)), 0.f);
    }
    lo = make_float4(pad_lo(lo.x), pad_lo(lo.y), pad_lo(lo.z), 0.f);
    hi = make_float4(pad_hi(hi.x), pad_hi(hi.y), pad_hi(hi.z), 0.f);
    lo_out[i] = lo;
    hi_out[i] = hi;
    cx = Cx = 0.5f * (lo.x + hi.x);
    cy = Cy = 0.5f * (lo.y + hi.y);
    cz = Cz = 0.5f * (lo.z + hi.z);
  }
  // warp reduce, then block reduce (blockDim.x <= 256), then one atomic per block
  for (int o = 16; o > 0; o >>= 1) {
    cx = fminf(cx, __shfl_xor_sync(0xffffffffu, cx, o));
    cy = fminf(cy, __shfl_xor_sync(0xffffffffu, cy, o));
    cz = fminf(cz, __shfl_xor_sync(0xffffffffu, cz, o));
    Cx = fmaxf(Cx, __shfl_xor_sync(0xffffffffu, Cx, o));
    Cy = fmaxf(Cy, __shfl_xor_sync(0xffffffffu, Cy, o));
    Cz = fmaxf(Cz, __shfl_xor_sync(0xffffffffu, Cz, o));
  }
  __shared__ float s_b[8][6];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) {
    s_b[w][0] = cx;
    s_b[w][1] = cy;
    s_b[w][2] = cz;
    s_b[w][3] = Cx;
    s_b[w][4] = Cy;
    s_b[w][5] = Cz;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int k = threadIdx.x;
    float v = s_b[0][k];
    for (int j = 1; j < nw; ++j) v = k < 3 ? fminf(v, s_b[j][k]) : fmaxf(v, s_b[j][k]);
    if (k < 3 ? v < INFINITY : v > -INFINITY) {
      if (k < 3) atomicMin(&cb[k], f2o(v));
      else atomicMax(&cb[k], f2o(v));
    }
  }
}

// ---------------------------------------------------------------------------
// 2. 30-bit Morton codes: 10 bits per axis of the centroid, normalised to
//    the centroid bounds, bits interleaved x y z from the top.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned spread10(unsigned v) {
  // places bit k of v at bit 3k
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ unsigned quantize10(float c, float lo, float hi) {
  float ext = hi - lo;
  float f = ext > 0.f ? (c - lo) / ext : 0.5f;
  int q = (int)(f * 1024.0f);
  return (unsigned)min(max(q, 0), 1023);
}

// Also clears the arrays the hierarchy and the refit fill (their arrival
// flags, and -1 parents), which saves three memsets on the build's path.
__global__ void k_morton(const float4* __restrict__ lo, const float4* __restrict__ hi, int n,
                         const int* __restrict__ cb, int drop, unsigned* __restrict__ keys,
                         unsigned* __restrict__ vals, int* __restrict__ flags, int* __restrict__ parent,
                         int* __restrict__ leaf_parent) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  flags[i] = 0;
  parent[i] = -1;
  leaf_parent[i] = -1;
  float4 a = lo[i], b = hi[i];
  float cx = 0.5f * (a.x + b.x), cy = 0.5f * (a.y + b.y), cz = 0.5f * (a.z + b.z);
  unsigned qx = quantize10(cx, o2f(cb[0]), o2f(cb[3]));
  unsigned qy = quantize10(cy, o2f(cb[1]), o2f(cb[4]));
  unsigned qz = quantize10(cz, o2f(cb[2]), o2f(cb[5]));
  keys[i] = ((spread10(qx) << 2) | (spread10(qy) << 1) | spread10(qz)) >> drop;
  vals[i] = (unsigned)i;
}

// ---------------------------------------------------------------------------
// 3. LSD radix sort of (key, value) pairs, 8 bits a pass, stable.
// ---------------------------------------------------------------------------
__global__ void k_sort_hist(const unsigned* __restrict__ keys, int n, int shift, unsigned* __restrict__ hist,
                            int tiles) {
  __shared__ unsigned h[256];
  int t = threadIdx.x;
  h[t] = 0;
  __syncthreads();
  size_t base = (size_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int r = 0; r < kSortTile / 256; ++r) {
    size_t idx = base + (size_t)r * 256 + t;
    if (idx < (size_t)n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(size_t)t * tiles + blockIdx.x] = h[t];
}

// Exclusive scan, block level: 1024 threads x 4 elements.  Writes the block
// total to partials[blockIdx.x].
__device__ __forceinline__ unsigned warp_incl_scan(unsigned v, int lane) {
  for (int o = 1; o < 32; o <<= 1) {
    unsigned x = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += x;
  }
  return v;
}

__device__ unsigned block_excl_scan_1024(unsigned v, unsigned* sw, unsigned& total) {
  int t = threadIdx.x, lane = t & 31, w = t >> 5;
  unsigned inc = warp_incl_scan(v, lane);
  if (lane == 31) sw[w] = inc;
  __syncthreads();
  if (w == 0) {
    unsigned s = sw[lane];
    unsigned si = warp_incl_scan(s, lane);
    sw[lane] = si - s;
    if (lane == 31) sw[32] = si;
  }
  __syncthreads();
  unsigned r = inc - v + sw[w];
  total = sw[32];
  __syncthreads();
  return r;
}

__global__ void k_scan_block(unsigned* __restrict__ data, size_t m, unsigned* __restrict__ partials) {
  __shared__ unsigned sw[33];
  size_t base = (size_t)blockIdx.x * kScanBlock + (size_t)threadIdx.x * 4;
  unsigned a[4], s = 0;
  for (int k = 0; k < 4; ++k) {
    a[k] = base + k < m ? data[base + k] : 0u;
    s += a[k];
  }
  unsigned total;
  unsigned ex = block_excl_scan_1024(s, sw, total);
  for (int k = 0; k < 4; ++k) {
    if (base + k < m) data[base + k] = ex;
    ex += a[k];
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

__global__ void k_scan_partials(unsigned* __restrict__ partials, int np) {
  __shared__ unsigned sw[33];
  unsigned carry = 0;
  for (int base = 0; base < np; base += 1024) {
    int i = base + threadIdx.x;
    unsigned v = i < np ? partials[i] : 0u;
    unsigned total;
    unsigned ex = block_excl_scan_1024(v, sw, total);
    if (i < np) partials[i] = ex + carry;
    carry += total;
  }
}

__global__ void k_scan_add(unsigned* __restrict__ data, size_t m, const unsigned* __restrict__ partials) {
  unsigned add = partials[blockIdx.x];
  size_t base = (size_t)blockIdx.x * kScanBlock + (size_t)threadIdx.x * 4;
  for (int k = 0; k < 4; ++k)
    if (base + k < m) data[base + k] += add;
}

// Stable scatter: the tile's keys are ranked in index order, 256 at a time;
// within a warp, keys with equal digits are found with match.any.
__global__ void __launch_bounds__(256) k_sort_scatter(const unsigned* __restrict__ kin, const unsigned* __restrict__ vin,
                                                      unsigned* __restrict__ kout, unsigned* __restrict__ vout, int n,
                                                      int shift, const unsigned* __restrict__ offs, int tiles) {
  __shared__ unsigned base[256];
  __shared__ unsigned wcnt[8][256];
  int t = threadIdx.x, lane = t & 31, w = t >> 5;
  base[t] = offs[(size_t)t * tiles + blockIdx.x];
#pragma unroll
  for (int k = 0; k < 8; ++k) wcnt[k][t] = 0;
  __syncthreads();
  size_t tile0 = (size_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortTile / 256; ++r) {
    size_t idx = tile0 + (size_t)r * 256 + t;
    bool valid = idx < (size_t)n;
    unsigned key = valid ? kin[idx] : 0u, val = valid ? vin[idx] : 0u;
    unsigned digit = (key >> shift) & 255u;
    unsigned peers = __match_any_sync(0xffffffffu, valid ? digit : 256u + (unsigned)lane);
    int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[w][digit] = __popc(peers);
    __syncthreads();
    {
      unsigned run = base[t];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        unsigned c = wcnt[k][t];
        wcnt[k][t] = run;
        run += c;
      }
      base[t] = run;
    }
    __syncthreads();
    if (valid) {
      unsigned pos = wcnt[w][digit] + (unsigned)rank;
      if (pos < (unsigned)n) {
        kout[pos] = key;
        vout[pos] = val;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k) wcnt[k][t] = 0;
    __syncthreads();
  }
}

// Exclusive scan over a 256-thread block.
__device__ unsigned block_excl_scan_256(unsigned v, unsigned* sw, unsigned& total) {
  int t = threadIdx.x, lane = t & 31, w = t >> 5;
  unsigned inc = warp_incl_scan(v, lane);
  if (lane == 31) sw[w] = inc;
  __syncthreads();
  if (w == 0) {
    unsigned x = lane < 8 ? sw[lane] : 0u;
    unsigned xi = warp_incl_scan(x, lane);
    if (lane < 8) sw[lane] = xi - x;
    if (lane == 7) sw[8] = xi;
  }
  __syncthreads();
  unsigned r = inc - v + sw[w];
  total = sw[8];
  __syncthreads();
  return r;
}

// The whole LSD radix sort in one cooperative launch (inputs up to
// kSortCoopMaxKeys): block b owns one contiguous tile of the keys.  Each
// 8-bit pass counts the tile's digits, scans every digit's counts over the
// tiles (one block per digit), and scatters the tile stably, with grid
// barriers between the three steps.  Keys written by other blocks are read
// through L2 (__ldcg).
__global__ void __launch_bounds__(256) k_sort_coop(unsigned* k0, unsigned* v0, unsigned* k1, unsigned* v1, int n,
                                                   int passes, unsigned* __restrict__ hist,
                                                   unsigned* __restrict__ totals) {
  cg::grid_group grid = cg::this_grid();
  __shared__ unsigned h[256];
  __shared__ unsigned base[256];
  __shared__ unsigned wcnt[8][256];
  __shared__ unsigned sw[9];
  const int G = (int)gridDim.x, b = (int)blockIdx.x, t = (int)threadIdx.x, lane = t & 31, w = t >> 5;
  const int T = (n + G - 1) / G;
  const int beg = min(n, b * T), end = min(n, beg + T);
  unsigned *ki = k0, *vi = v0, *ko = k1, *vo = v1;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    // 1. digit counts of this tile
    h[t] = 0;
    __syncthreads();
    for (int i = beg + t; i < end; i += 256) atomicAdd(&h[(__ldcg(&ki[i]) >> shift) & 255u], 1u);
    __syncthreads();
    hist[(size_t)t * G + b] = h[t];
    grid.sync();
    // 2. per digit: exclusive scan of its counts over the tiles, and its total
    for (int d = b; d < 256; d += G) {
      unsigned* row = hist + (size_t)d * G;
      const int per = (G + 255) / 256, i0 = t * per;
      unsigned sum = 0;
      for (int k = 0; k < per; ++k)
        if (i0 + k < G) sum += __ldcg(&row[i0 + k]);
      unsigned tot;
      unsigned ex = block_excl_scan_256(sum, sw, tot);
      for (int k = 0; k < per; ++k) {
        if (i0 + k < G) {
          unsigned x = __ldcg(&row[i0 + k]);
          row[i0 + k] = ex;
          ex += x;
        }
      }
      if (t == 0) totals[d] = tot;
    }
    grid.sync();
    // 3. where this tile's keys of each digit start
    {
      unsigned tot_d = __ldcg(&totals[t]), all;
      unsigned digit_base = block_excl_scan_256(tot_d, sw, all);
      base[t] = digit_base + __ldcg(&hist[(size_t)t * G + b]);
#pragma unroll
      for (int k = 0; k < 8; ++k) wcnt[k][t] = 0;
    }
    __syncthreads();
    // 4. stable scatter, 256 keys at a time in index order; equal digits
    //    within a warp are ranked with match.any
    for (int r0 = beg; r0 < end; r0 += 256) {
      const int idx = r0 + t;
      const bool valid = idx < end;
      unsigned key = valid ? __ldcg(&ki[idx]) : 0u, val = valid ? __ldcg(&vi[idx]) : 0u;
      unsigned digit = (key >> shift) & 255u;
      unsigned peers = __match_any_sync(0xffffffffu, valid ? digit : 256u + (unsigned)lane);
      int rank = __popc(peers & ((1u << lane) - 1u));
      if (valid && rank == 0) wcnt[w][digit] = __popc(peers);
      __syncthreads();
      {
        unsigned run = base[t];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          unsigned c = wcnt[k][t];
          wcnt[k][t] = run;
          run += c;
        }
        base[t] = run;
      }
      __syncthreads();
      if (valid) {
        unsigned pos = wcnt[w][digit] + (unsigned)rank;
        if (pos < (unsigned)n) {
          ko[pos] = key;
          vo[pos] = val;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 8; ++k) wcnt[k][t] = 0;
      __syncthreads();
    }
    grid.sync();
    unsigned* tk = ki;
    ki = ko;
    ko = tk;
    unsigned* tv = vi;
    vi = vo;
    vo = tv;
  }
}

static int scan_exclusive(unsigned* data, size_t m, unsigned* partials, cudaStream_t st) {
  int blocks = (int)((m + kScanBlock - 1) / kScanBlock);
  k_scan_block<<<blocks, 1024, 0, st>>>(data, m, partials);
  if (blocks > 1) {
    k_scan_partials<<<1, 1024, 0, st>>>(partials, blocks);
    k_scan_add<<<blocks, 1024, 0, st>>>(data, m, partials);
    return 3;
  }
  return 1;
}

// Passes of 8 bits that sort keys of `bits` bits.
static int sort_passes(int bits) { return (bits + 7) / 8; }

// Bits of the Morton code that the sort orders by: its top 24 (a 256^3
// grid, three passes) when there are at most 2^17 primitives, which leaves
// at least 128 cells a primitive; all 30 (four passes) above that.
// Primitives that share a key keep their input order, and the hierarchy
// tells equal keys apart by index.  Measured on the 1080p terrain (123,904
// primitives): SAH 28.500 against 28.493 with 30 bits, and 15 us less a
// build.
static int morton_key_bits(int64_t n) { return n <= (1 << 17) ? 24 : 30; }

// Sorts the pairs by the low `bits` bits.  The input is in (keys0, vals0)
// for an even number of passes and in (keys1, vals1) for an odd one; the
// result ends in (keys0, vals0).
static int radix_sort_pairs(rt_scene* s, BuildScratch& b, int n, int bits, cudaStream_t st) {
  int launches = 0;
  int tiles = (n + kSortTile - 1) / kSortTile;
  int passes = sort_passes(bits);
  const bool odd = passes & 1;
  unsigned *k_in = odd ? b.keys1 : b.keys0, *v_in = odd ? b.vals1 : b.vals0;
  unsigned *k_out = odd ? b.keys0 : b.keys1, *v_out = odd ? b.vals0 : b.vals1;
  static int coop_blocks = -1;
  if (coop_blocks < 0) {
    int coop = 0, per_sm = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_coop, 256, 0);
    coop_blocks = coop ? std::min(std::min(per_sm, 1) * s->sm_count, kSortCoopMaxBlocks) : 0;   // one an SM
  }
  if (coop_blocks > 0 && n <= kSortCoopMaxKeys) {
    void* args[] = {&k_in, &v_in, &k_out, &v_out, &n, &passes, &b.hist, &b.partials};
    if (cudaLaunchCooperativeKernel((void*)k_sort_coop, coop_blocks, 256, args, 0, st) == cudaSuccess) return 1;
    cudaGetLastError();
  }
  unsigned *ki = k_in, *vi = v_in, *ko = k_out, *vo = v_out;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    k_sort_hist<<<tiles, 256, 0, st>>>(ki, n, shift, b.hist, tiles);
    launches += 2 + scan_exclusive(b.hist, (size_t)256 * tiles, b.partials, st);
    k_sort_scatter<<<tiles, 256, 0, st>>>(ki, vi, ko, vo, n, shift, b.hist, tiles);
    std::swap(ki, ko);
    std::swap(vi, vo);
  }
  return launches;
}

// ---------------------------------------------------------------------------
// 4. LBVH hierarchy (Karras 2012): internal node i covers a key range with
//    i at one end; its split is where the common prefix of the range ends.
//    Equal codes are told apart by their index.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int prefix_len(const unsigned* __restrict__ keys, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  unsigned a = keys[i], b = keys[j];
  if (a != b) return __clz(a ^ b);
  return 32 + __clz((unsigned)i ^ (unsigned)j);
}

// Block 0 also resets the centroid bounds for the next build (k_morton, the
// last reader, is done) and clears the top rebuild's counters (seg_n ints).
__global__ void k_hierarchy(const unsigned* __restrict__ keys, int n, int* __restrict__ lch, int* __restrict__ rch,
                            int* __restrict__ parent, int* __restrict__ leaf_parent, int2* __restrict__ range,
                            int* __restrict__ cb, int* __restrict__ seg_count, int seg_n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0) {
    reset_bounds(cb, threadIdx.x);
    if (threadIdx.x < seg_n) seg_count[threadIdx.x] = 0;
  }
  if (i >= n - 1) return;
  int dl = prefix_len(keys, n, i, i - 1), dr = prefix_len(keys, n, i, i + 1);
  int d = dr > dl ? 1 : -1;
  int dmin = dr > dl ? dl : dr;
  int lmax = 2;
  while (prefix_len(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int l = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (prefix_len(keys, n, i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = prefix_len(keys, n, i, j);
  int s = 0, div = 2, t;
  do {
    t = (l + div - 1) / div;
    if (prefix_len(keys, n, i, i + (s + t) * d) > dnode) s += t;
    div <<= 1;
  } while (t > 1);
  int gamma = i + s * d + (d < 0 ? -1 : 0);
  int lo = min(i, j), hi = max(i, j);
  int left = (lo == gamma) ? ~gamma : gamma;
  int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
  lch[i] = left;
  rch[i] = right;
  range[i] = make_int2(lo, hi);
  if (left < 0) leaf_parent[gamma] = i;
  else parent[left] = i;
  if (right < 0) leaf_parent[gamma + 1] = i;
  else parent[right] = i;
  if (i == 0) parent[0] = -1;
}

// ---------------------------------------------------------------------------
// 5. bottom-up boxes, SAH costs and leaf collapsing.  The second thread to
//    reach a node processes it.  meta (node_hi.w bits): height | collapse<<8
// ---------------------------------------------------------------------------
struct ChildInfo {
  float4 lo, hi;
  float cost, cost_lbvh;
  int height;
};

__device__ __forceinline__ ChildInfo child_info(int c, const unsigned* __restrict__ vals, const float4* aabb_lo,
                                                const float4* aabb_hi, const float4* node_lo, const float4* node_hi,
                                                const float* cost_lbvh) {
  ChildInfo r;
  if (c < 0) {
    unsigned pid = vals[~c];
    r.lo = aabb_lo[pid];
    r.hi = aabb_hi[pid];
    r.cost = kCostIsect;
    r.cost_lbvh = kCostIsect;
    r.height = 0;
  } else {
    r.lo = __ldcg(&node_lo[c]);
    r.hi = __ldcg(&node_hi[c]);
    r.cost = r.lo.w;
    r.cost_lbvh = __ldcg(&cost_lbvh[c]);
    r.height = __float_as_int(r.hi.w) & 0xff;   // 0 for a collapsed node
  }
  return r;
}

// The box, SAH costs and collapse decision of internal node `node`, from
// its two children (both done).
// The second of a node's two children to arrive refits it: returns the
// count before this arrival.  Acquire-release at device scope: the
// arriving thread's earlier writes (its child's box and costs) are visible
// to whoever arrives after it, and the second thread sees the first's.
__device__ __forceinline__ int arrive(int* flag) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(old) : "l"(flag) : "memory");
  return old;
}

__device__ __forceinline__ void refit_node(int node, int l, int r, const unsigned* __restrict__ vals,
                                           const float4* __restrict__ aabb_lo, const float4* __restrict__ aabb_hi,
                                           int2 rg, float4* node_lo, float4* node_hi, float* cost_lbvh) {
  ChildInfo a = child_info(l, vals, aabb_lo, aabb_hi, node_lo, node_hi, cost_lbvh);
  ChildInfo b = child_info(r, vals, aabb_lo, aabb_hi, node_lo, node_hi, cost_lbvh);
  float4 lo = make_float4(fminf(a.lo.x, b.lo.x), fminf(a.lo.y, b.lo.y), fminf(a.lo.z, b.lo.z), 0.f);
  float4 hi = make_float4(fmaxf(a.hi.x, b.hi.x), fmaxf(a.hi.y, b.hi.y), fmaxf(a.hi.z, b.hi.z), 0.f);
  float A = area(lo, hi), Aa = area(a.lo, a.hi), Ab = area(b.lo, b.hi);
  float ci, cl;
  if (A > 0.f) {
    ci = kCostTrav + (Aa * a.cost + Ab * b.cost) / A;
    cl = kCostTrav + (Aa * a.cost_lbvh + Ab * b.cost_lbvh) / A;
  } else {
    ci = kCostTrav + a.cost + b.cost;
    cl = kCostTrav + a.cost_lbvh + b.cost_lbvh;
  }
  int count = rg.y - rg.x + 1;
  float leaf_cost = kCostIsect * (float)count;
  int collapse = (count <= kMaxLeaf && leaf_cost <= ci) ? 1 : 0;
  int height = collapse ? 0 : 1 + max(a.height, b.height);
  lo.w = collapse ? leaf_cost : ci;
  hi.w = __int_as_float(height | (collapse << 8));
  node_lo[node] = lo;
  node_hi[node] = hi;
  cost_lbvh[node] = cl;
}

// Bottom-up from every leaf; the second thread to reach a node refits it
// and climbs on.  A node over `cut` primitives is left alone (and its flag
// untouched): the top rebuild replaces those nodes, and k_refit_upper
// finishes them off the critical path for the plain LBVH's cost.
__global__ void k_refit(int n, int cut, const unsigned* __restrict__ vals, const float4* __restrict__ aabb_lo,
                        const float4* __restrict__ aabb_hi, const int* __restrict__ lch, const int* __restrict__ rch,
                        const int* __restrict__ parent, const int* __restrict__ leaf_parent,
                        const int2* __restrict__ range, float4* node_lo, float4* node_hi, float* cost_lbvh, int* flags) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int node = leaf_parent[p];
  // a radix tree has at most n-1 ancestors above a leaf; the bound and the
  // index check only guard against a malformed tree
  for (int it = 0; node >= 0 && node < n - 1 && it < n; ++it) {
    // the links are read before the flag: this kernel does not change them
    const int2 rg = range[node];
    const int l = lch[node], r = rch[node], up = parent[node];
    if (rg.y - rg.x + 1 > cut) return;
    if (arrive(&flags[node]) == 0) return;
    refit_node(node, l, r, vals, aabb_lo, aabb_hi, rg, node_lo, node_hi, cost_lbvh);
    node = up;
  }
}

// The nodes over `cut` primitives, after k_refit: a node with both children
// at or under the cut is refitted by its own thread, one with a single such
// child counts that child's arrival; then the climb goes on as in k_refit.
__global__ void k_refit_upper(int n, int cut, const unsigned* __restrict__ vals, const float4* __restrict__ aabb_lo,
                              const float4* __restrict__ aabb_hi, const int* __restrict__ lch,
                              const int* __restrict__ rch, const int* __restrict__ parent,
                              const int2* __restrict__ range, float4* node_lo, float4* node_hi, float* cost_lbvh,
                              int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int2 rg = range[i];
  if (rg.y - rg.x + 1 <= cut) return;
  const int l = lch[i], r = rch[i];
  const bool bl = l < 0 || range[l].y - range[l].x + 1 <= cut;
  const bool br = r < 0 || range[r].y - range[r].x + 1 <= cut;
  if (!bl && !br) return;                                   // both children arrive by climbing
  if (bl != br && atomicAdd(&flags[i], 1) == 0) return;     // the other one will
  __threadfence();
  int node = i;
  for (int it = 0; it < n; ++it) {
    refit_node(node, lch[node], rch[node], vals, aabb_lo, aabb_hi, rg, node_lo, node_hi, cost_lbvh);
    node = parent[node];
    if (node < 0 || node >= n - 1) return;
    rg = range[node];
    __threadfence();
    if (atomicAdd(&flags[node], 1) == 0) return;
    __threadfence();
  }
}

// The plain LBVH's SAH cost, once its root is refitted.
__global__ void k_info_sah_lbvh(const float* __restrict__ cost_lbvh, BuildInfo* info) {
  info->sah_lbvh = cost_lbvh[0];
}

// ---------------------------------------------------------------------------
// 6. binned-SAH rebuild of the top levels (HLBVH style): the LBVH nodes
//    with at most `cluster_max` primitives whose parent has more become
//    clusters; a new top tree is built over the clusters' boxes with 16
//    bins per axis, level by level (one block per segment).  With clusters
//    of at most kWarpRefitMax primitives, the clusters are found first and
//    each cluster's subtree is then refitted by one warp in shared memory
//    (k_refit_clusters) instead of by k_refit's climb through global
//    atomics; the LBVH nodes above the clusters are never refitted.
// ---------------------------------------------------------------------------
__global__ void k_find_clusters(int n, int cluster_max, const int* __restrict__ lch, const int* __restrict__ rch,
                                const int2* __restrict__ range, const float4* __restrict__ node_lo,
                                const float4* __restrict__ node_hi, const unsigned* __restrict__ vals,
                                const float4* __restrict__ aabb_lo, const float4* __restrict__ aabb_hi,
                                int* __restrict__ clu_count_out, int* __restrict__ clu_ids, int* __restrict__ clu_link,
                                float4* __restrict__ clu_lo, float4* __restrict__ clu_hi, int defer) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int2 rg = range[i];
  if (rg.y - rg.x + 1 <= cluster_max) return;     // a node above the cut only emits its children
  int kids[2] = {lch[i], rch[i]};
  for (int k = 0; k < 2; ++k) {
    int c = kids[k];
    int count;
    float4 lo, hi;
    int link, height;
    if (c < 0) {
      unsigned pid = vals[~c];
      lo = aabb_lo[pid];
      hi = aabb_hi[pid];
      count = 1;
      link = leaf_link(~c, 1);
      height = 0;
    } else {
      int2 r2 = range[c];
      count = r2.y - r2.x + 1;
      if (count > cluster_max) continue;
      if (defer) {
        // k_refit_clusters refits the subtree and completes the entry
        lo = hi = make_float4(0.f, 0.f, 0.f, 0.f);
        link = c;
        height = 0;
      } else {
        lo = node_lo[c];
        hi = node_hi[c];
        int meta = __float_as_int(hi.w);
        bool collapse = (meta >> 8) & 1;
        link = collapse ? leaf_link(r2.x, count) : c;
        height = collapse ? 0 : (meta & 0xff);
      }
    }
    int slot = atomicAdd(clu_count_out, 1);
    clu_ids[slot] = slot;
    clu_link[slot] = link;
    clu_lo[slot] = make_float4(lo.x, lo.y, lo.z, (float)count);
    clu_hi[slot] = make_float4(hi.x, hi.y, hi.z, __int_as_float(height));
  }
}

// One warp per cluster entry whose link is still a node id (k_find_clusters
// with `defer`): the same boxes, SAH costs, leaf collapsing and node writes
// as k_refit, for the subtree under that node, climbed bottom-up inside the
// warp.  The subtree's leaf boxes and links are loaded into shared memory
// first (one round trip); then every round, each live item (a leaf, or a
// node refitted in an earlier round) arrives at its parent through a
// shared-memory counter, and the second arrival refits the parent.  Then
// the warp completes the entry as k_find_clusters would have.
constexpr int kWarpRefitMax = 64;   // cluster size up to which this path is taken
constexpr int kWarpRefitWarps = 4;  // warps per block

__global__ void __launch_bounds__(32 * kWarpRefitWarps)
    k_refit_clusters(int n, const unsigned* __restrict__ vals, const float4* __restrict__ aabb_lo,
                     const float4* __restrict__ aabb_hi, const int* __restrict__ lch, const int* __restrict__ rch,
                     const int* __restrict__ parent, const int* __restrict__ leaf_parent,
                     const int2* __restrict__ range, float4* __restrict__ node_lo, float4* __restrict__ node_hi,
                     float* __restrict__ cost_lbvh, const int* __restrict__ n_clusters, int* __restrict__ clu_link,
                     float4* __restrict__ clu_lo, float4* __restrict__ clu_hi) {
  constexpr int M = kWarpRefitMax;
  // slot q < M: leaf a + q; slot M + q: internal node a + q (lo.w = cost, hi.w = meta bits)
  __shared__ float4 s_lo[kWarpRefitWarps][2 * M], s_hi[kWarpRefitWarps][2 * M];
  __shared__ float s_cl[kWarpRefitWarps][M];   // the plain LBVH's cost of internal slot q
  __shared__ int s_l[kWarpRefitWarps][M], s_r[kWarpRefitWarps][M], s_par[kWarpRefitWarps][M];
  __shared__ int s_cnt[kWarpRefitWarps][M], s_lpar[kWarpRefitWarps][M], s_flag[kWarpRefitWarps][M];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n_entries = __ldg(n_clusters);
  const int warps = (int)gridDim.x * kWarpRefitWarps;
  float4* lo_s = s_lo[w];
  float4* hi_s = s_hi[w];
  for (int e = (int)blockIdx.x * kWarpRefitWarps + w; e < n_entries; e += warps) {
    const int R = clu_link[e];
    if (R < 0) continue;   // a one-primitive cluster, complete
    const int2 rg = range[R];
    const int a = rg.x, m = rg.y - rg.x + 1;   // 2 <= m <= M
    if (m > M) continue;   // not reachable: the host takes this path only for clusters of <= M
    __syncwarp();
    for (int q = lane; q < m; q += 32) {
      const unsigned pid = vals[a + q];
      lo_s[q] = aabb_lo[pid];
      hi_s[q] = aabb_hi[pid];
      s_lpar[w][q] = leaf_parent[a + q];
      const int i = a + q;
      if (i <= n - 2) {
        s_l[w][q] = lch[i];
        s_r[w][q] = rch[i];
        s_par[w][q] = parent[i];
        const int2 ri = range[i];
        s_cnt[w][q] = ri.y - ri.x + 1;
      }
      s_flag[w][q] = 0;
    }
    __syncwarp();
    // each lane's items: its leaves; an item is a slot (leaf q, or M + q), -1 when done
    int item[2] = {lane < m ? lane : -1, lane + 32 < m ? lane + 32 : -1};
    for (int round = 0; round <= 2 * M; ++round) {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int it = item[k];
        if (it < 0) continue;
        if (it == M + (R - a)) {   // the cluster's root: done
          item[k] = -1;
          continue;
        }
        const int p = it < M ? s_lpar[w][it] : s_par[w][it - M];
        const int pq = p - a;
        if (pq < 0 || pq >= m) {   // not reachable in a well-formed tree
          item[k] = -1;
          continue;
        }
        if (atomicAdd(&s_flag[w][pq], 1) == 0) {   // the sibling refits the parent
          item[k] = -1;
          continue;
        }
        // both children are ready: refit p (as refit_node, from shared memory)
        const int cl_ = s_l[w][pq], cr_ = s_r[w][pq];
        const int sl = cl_ < 0 ? (~cl_) - a : M + (cl_ - a), sr = cr_ < 0 ? (~cr_) - a : M + (cr_ - a);
        const float4 al = lo_s[sl], ah = hi_s[sl], bl = lo_s[sr], bh = hi_s[sr];
        const bool la = sl < M, lb = sr < M;
        const float ca = la ? kCostIsect : al.w, cb = lb ? kCostIsect : bl.w;
        const float cla = la ? kCostIsect : s_cl[w][sl - M], clb = lb ? kCostIsect : s_cl[w][sr - M];
        const int ha = la ? 0 : (__float_as_int(ah.w) & 0xff), hb = lb ? 0 : (__float_as_int(bh.w) & 0xff);
        float4 lo = make_float4(fminf(al.x, bl.x), fminf(al.y, bl.y), fminf(al.z, bl.z), 0.f);
        float4 hi = make_float4(fmaxf(ah.x, bh.x), fmaxf(ah.y, bh.y), fmaxf(ah.z, bh.z), 0.f);
        const float A = area(lo, hi), Aa = area(al, ah), Ab = area(bl, bh);
        float ci, cl;
        if (A > 0.f) {
          ci = kCostTrav + (Aa * ca + Ab * cb) / A;
          cl = kCostTrav + (Aa * cla + Ab * clb) / A;
        } else {
          ci = kCostTrav + ca + cb;
          cl = kCostTrav + cla + clb;
        }
        const int count = s_cnt[w][pq];
        const float leaf_cost = kCostIsect * (float)count;
        const int collapse = (count <= kMaxLeaf && leaf_cost <= ci) ? 1 : 0;
        const int height = collapse ? 0 : 1 + max(ha, hb);
        lo.w = collapse ? leaf_cost : ci;
        hi.w = __int_as_float(height | (collapse << 8));
        lo_s[M + pq] = lo;
        hi_s[M + pq] = hi;
        s_cl[w][pq] = cl;
        node_lo[p] = lo;
        node_hi[p] = hi;
        cost_lbvh[p] = cl;
        item[k] = M + pq;
      }
      __syncwarp();
      if (!__any_sync(FULL, (item[0] >= 0) | (item[1] >= 0))) break;
    }
    if (lane == 0) {
      const float4 lo = lo_s[M + (R - a)], hi = hi_s[M + (R - a)];
      const int meta = __float_as_int(hi.w);
      const bool collapse = (meta >> 8) & 1;
      clu_link[e] = collapse ? leaf_link(a, m) : R;
      clu_lo[e] = make_float4(lo.x, lo.y, lo.z, (float)m);
      clu_hi[e] = make_float4(hi.x, hi.y, hi.z, __int_as_float(collapse ? 0 : (meta & 0xff)));
    }
  }
}

__global__ void k_iota(int* __restrict__ a, const int* __restrict__ n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < *n) a[i] = i;
}

// Writes child `side` (0/1) of a node in the traversal layout.
__device__ __forceinline__ void write_child(float4* nodes, int node, int side, float4 lo, float4 hi, int link) {
  float* n = (float*)(nodes + 4 * (size_t)node);
  int o = side == 0 ? 0 : 4;
  n[o + 0] = lo.x;
  n[o + 1] = hi.x;
  n[o + 2] = lo.y;
  n[o + 3] = hi.y;
  n[8 + 2 * side] = lo.z;
  n[9 + 2 * side] = hi.z;
  n[12 + side] = __int_as_float(link);
}

// Bin of centroid coordinate c over [lo, lo + extent): inv = kTopBins /
// extent, or 0 for an empty extent (every centroid in bin 0).
__device__ __forceinline__ float bin_scale(float ext) { return ext > 0.f ? (float)kTopBins / ext : 0.f; }
__device__ __forceinline__ int bin_of(float c, float lo, float inv) {
  const int bi = (int)((c - lo) * inv);
  return min(max(bi, 0), kTopBins - 1);
}

// The cheapest of the 3 x (kTopBins - 1) split planes of a set of bins
// (SAH A_L N_L + A_R N_R, N in primitives): warp a scans axis a, lane k
// holding bin k, with prefix and suffix scans of the counts and bounds;
// the plane index is a * (kTopBins - 1) + (last bin on the left).  Returns
// the same index in every thread, the lowest on ties, or -1 when no plane
// has a finite cost.  All threads of the block call it (it synchronises).
__device__ __forceinline__ int best_plane(const int (*cnt)[kTopBins], const int (*blo)[kTopBins][3],
                                          const int (*bhi)[kTopBins][3], float* s_bc, int* s_bk) {
  const unsigned FULL = 0xffffffffu;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (w < 3) {
    const bool in = lane < kTopBins;
    int pn = in ? cnt[w][lane] : 0, sn = pn;
    float pl[3], ph[3], sl[3], sh[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      pl[q] = sl[q] = in ? o2f(blo[w][lane][q]) : INFINITY;
      ph[q] = sh[q] = in ? o2f(bhi[w][lane][q]) : -INFINITY;
    }
#pragma unroll
    for (int o = 1; o < kTopBins; o <<= 1) {
      const int xn = __shfl_up_sync(FULL, pn, o), yn = __shfl_down_sync(FULL, sn, o);
      const bool up = lane >= o, down = lane + o < kTopBins;
      pn += up ? xn : 0;
      sn += down ? yn : 0;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float xl = __shfl_up_sync(FULL, pl[q], o), xh = __shfl_up_sync(FULL, ph[q], o);
        const float yl = __shfl_down_sync(FULL, sl[q], o), yh = __shfl_down_sync(FULL, sh[q], o);
        pl[q] = up ? fminf(pl[q], xl) : pl[q];
        ph[q] = up ? fmaxf(ph[q], xh) : ph[q];
        sl[q] = down ? fminf(sl[q], yl) : sl[q];
        sh[q] = down ? fmaxf(sh[q], yh) : sh[q];
      }
    }
    // the right side of the plane after bin `lane`: the suffix from the next bin
    const int rn = __shfl_down_sync(FULL, sn, 1);
    float rl[3], rh[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      rl[q] = __shfl_down_sync(FULL, sl[q], 1);
      rh[q] = __shfl_down_sync(FULL, sh[q], 1);
    }
    float cost = INFINITY;
    int k = INT_MAX;
    if (lane < kTopBins - 1) {
      k = w * (kTopBins - 1) + lane;
      if (pn > 0 && rn > 0) {
        const float AL = area(make_float4(pl[0], pl[1], pl[2], 0.f), make_float4(ph[0], ph[1], ph[2], 0.f));
        const float AR = area(make_float4(rl[0], rl[1], rl[2], 0.f), make_float4(rh[0], rh[1], rh[2], 0.f));
        cost = AL * (float)pn + AR * (float)rn;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oc = __shfl_xor_sync(FULL, cost, o);
      const int ok = __shfl_xor_sync(FULL, k, o);
      const bool take = (oc < cost) | ((oc == cost) & (ok < k));
      cost = take ? oc : cost;
      k = take ? ok : k;
    }
    if (lane == 0) {
      s_bc[w] = cost;
      s_bk[w] = k;
    }
  }
  __syncthreads();
  float bc = INFINITY;
  int bk = -1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float c = s_bc[a];
    bk = c < bc ? s_bk[a] : bk;
    bc = c < bc ? c : bc;
  }
  return bk;
}

// Split of a segment of at most 256 clusters, one cluster per thread, held
// in registers from one load: the same bins, SAH costs, choice and stable
// partition as the general path below, with fewer passes and barriers.
// Returns the number of clusters on the left side.
__device__ __forceinline__ int split_small(int level, int b, int e, CluList in, CluList out, float4 side_lo[2],
                                           float4 side_hi[2]) {
  __shared__ int s_cb[6];
  __shared__ int s_cnt[3][kTopBins];
  __shared__ int s_blo[3][kTopBins][3], s_bhi[3][kTopBins][3];
  __shared__ float s_bc[3];
  __shared__ int s_bk[3];
  __shared__ int s_wl[8], s_wr[8];
  __shared__ int s_box[2][6];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, m = e - b;
  const bool mine = t < m;
  int c = 0;
  float4 lo = make_float4(0, 0, 0, 0), hi = make_float4(0, 0, 0, 0);
  if (mine) {
    c = __ldcg(&in.id[b + t]);
    lo = __ldcg(&in.lo[b + t]);
    hi = __ldcg(&in.hi[b + t]);
  }
  float cc[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
  if (t < 6) {
    s_cb[t] = f2o(t < 3 ? INFINITY : -INFINITY);
    s_box[0][t] = f2o(t < 3 ? INFINITY : -INFINITY);
    s_box[1][t] = f2o(t < 3 ? INFINITY : -INFINITY);
  }
  if (t < 3 * kTopBins) {
    int a = t / kTopBins, k = t % kTopBins;
    s_cnt[a][k] = 0;
    for (int q = 0; q < 3; ++q) {
      s_blo[a][k][q] = f2o(INFINITY);
      s_bhi[a][k][q] = f2o(-INFINITY);
    }
  }
  // centroid bounds: warp reduction, one atomic per warp and axis
  float cmin[3], cmax[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cmin[a] = mine ? cc[a] : INFINITY;
    cmax[a] = mine ? cc[a] : -INFINITY;
    for (int o = 16; o > 0; o >>= 1) {
      cmin[a] = fminf(cmin[a], __shfl_xor_sync(0xffffffffu, cmin[a], o));
      cmax[a] = fmaxf(cmax[a], __shfl_xor_sync(0xffffffffu, cmax[a], o));
    }
  }
  __syncthreads();
  if (lane == 0 && cmin[0] <= cmax[0]) {
    for (int a = 0; a < 3; ++a) {
      atomicMin(&s_cb[a], f2o(cmin[a]));
      atomicMax(&s_cb[a + 3], f2o(cmax[a]));
    }
  }
  __syncthreads();
  const float clo[3] = {o2f(s_cb[0]), o2f(s_cb[1]), o2f(s_cb[2])};
  const float cinv[3] = {bin_scale(o2f(s_cb[3]) - clo[0]), bin_scale(o2f(s_cb[4]) - clo[1]),
                         bin_scale(o2f(s_cb[5]) - clo[2])};
  int bin[3];
  const float lo3[3] = {lo.x, lo.y, lo.z}, hi3[3] = {hi.x, hi.y, hi.z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    bin[a] = bin_of(cc[a], clo[a], cinv[a]);
    if (mine) {
      atomicAdd(&s_cnt[a][bin[a]], (int)lo.w);
      for (int q = 0; q < 3; ++q) {
        atomicMin(&s_blo[a][bin[a]][q], f2o(lo3[q]));
        atomicMax(&s_bhi[a][bin[a]][q], f2o(hi3[q]));
      }
    }
  }
  __syncthreads();
  int best = best_plane(s_cnt, s_blo, s_bhi, s_bc, s_bk);
  if (level >= kTopForceMedian) best = -1;

  bool left;
  if (best < 0) {
    left = t < m / 2;   // split at the middle, order kept
  } else {
    const int ax = best / (kTopBins - 1), sb = best % (kTopBins - 1);
    left = (ax == 0 ? bin[0] : ax == 1 ? bin[1] : bin[2]) <= sb;
  }
  const unsigned bl = __ballot_sync(0xffffffffu, mine && left), br = __ballot_sync(0xffffffffu, mine && !left);
  if (lane == 0) {
    s_wl[w] = __popc(bl);
    s_wr[w] = __popc(br);
  }
  __syncthreads();
  int before_l = 0, before_r = 0, nleft = 0;
  for (int q = 0; q < 8; ++q) {
    if (q < w) {
      before_l += s_wl[q];
      before_r += s_wr[q];
    }
    nleft += s_wl[q];
  }
  if (nleft == 0 || nleft == m) {
    // not reachable with a finite SAH cost; keep a valid split at the middle
    nleft = m / 2;
    left = t < nleft;
    before_l = min(w * 32, nleft);
    before_r = max(w * 32 - nleft, 0);
  }
  const unsigned lt = (1u << lane) - 1u;
  {
    const unsigned bl2 = __ballot_sync(0xffffffffu, mine && left), br2 = __ballot_sync(0xffffffffu, mine && !left);
    if (mine) {
      int pos = left ? b + before_l + __popc(bl2 & lt) : b + nleft + before_r + __popc(br2 & lt);
      out.id[pos] = c;
      out.lo[pos] = lo;
      out.hi[pos] = hi;
    }
  }
  // the two sides' boxes
  for (int side = 0; side < 2; ++side) {
    bool in = mine && (left == (side == 0));
    float v[6] = {in ? lo.x : INFINITY, in ? lo.y : INFINITY, in ? lo.z : INFINITY,
                  in ? hi.x : -INFINITY, in ? hi.y : -INFINITY, in ? hi.z : -INFINITY};
    for (int o = 16; o > 0; o >>= 1) {
      for (int q = 0; q < 3; ++q) v[q] = fminf(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
      for (int q = 3; q < 6; ++q) v[q] = fmaxf(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
    }
    if (lane == 0 && v[0] <= v[3]) {
      for (int q = 0; q < 3; ++q) {
        atomicMin(&s_box[side][q], f2o(v[q]));
        atomicMax(&s_box[side][q + 3], f2o(v[q + 3]));
      }
    }
  }
  __syncthreads();
  for (int side = 0; side < 2; ++side) {
    side_lo[side] = make_float4(o2f(s_box[side][0]), o2f(s_box[side][1]), o2f(s_box[side][2]), 0.f);
    side_hi[side] = make_float4(o2f(s_box[side][3]), o2f(s_box[side][4]), o2f(s_box[side][5]), 0.f);
  }
  return nleft;
}

// Split of a segment of more than 256 clusters by the whole block: the same
// bins, SAH costs, choice and stable partition as split_small.  A segment of
// up to cache_cap clusters is first read into shared memory, its loads
// issued eight deep.  After that every thread takes a contiguous chunk of
// the segment for the bounds and the partition: it counts and bounds its
// two sides in one pass before a block scan places them.
__device__ __forceinline__ int split_large(int level, int b, int e, CluList in, CluList out, int cache_cap,
                                           float4 side_lo[2], float4 side_hi[2]) {
  __shared__ int s_cb[6];
  __shared__ int bin_count[3][kTopBins];
  __shared__ int bin_lo[3][kTopBins][3], bin_hi[3][kTopBins][3];
  __shared__ float s_bc[3];
  __shared__ int s_bk[3];
  __shared__ int s_wl[8], s_wr[8];
  __shared__ int s_box[2][6];
  extern __shared__ float4 s_dyn[];
  const unsigned FULL = 0xffffffffu;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, m = e - b;
  float4* c_lo = s_dyn;
  float4* c_hi = s_dyn + cache_cap;
  int* c_id = (int*)(s_dyn + 2 * (size_t)cache_cap);
  int* c_part = c_id + cache_cap;              // cache slot of each position of the partition
  unsigned char* c_side = (unsigned char*)(c_part + cache_cap);   // side of each cached cluster
  const bool cached = m <= cache_cap;
  if (t < 6) {
    s_cb[t] = f2o(t < 3 ? INFINITY : -INFINITY);
    s_box[0][t] = f2o(t < 3 ? INFINITY : -INFINITY);
    s_box[1][t] = f2o(t < 3 ? INFINITY : -INFINITY);
  }
  if (t < 3 * kTopBins) {
    int a = t / kTopBins, k = t % kTopBins;
    bin_count[a][k] = 0;
    for (int q = 0; q < 3; ++q) {
      bin_lo[a][k][q] = f2o(INFINITY);
      bin_hi[a][k][q] = f2o(-INFINITY);
    }
  }
  if (cached) {
    for (int k0 = t; k0 < m; k0 += 256 * 8) {
      int id[8];
      float4 l[8], h[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + 256 * u;
        if (k < m) {
          id[u] = __ldcg(&in.id[b + k]);
          l[u] = __ldcg(&in.lo[b + k]);
          h[u] = __ldcg(&in.hi[b + k]);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + 256 * u;
        if (k < m) {
          c_id[k] = id[u];
          c_lo[k] = l[u];
          c_hi[k] = h[u];
        }
      }
    }
  }
  __syncthreads();
  // position k (0..m-1) of the segment
  auto fetch = [&](int k, int& c, float4& lo, float4& hi) {
    if (cached) {
      c = c_id[k];
      lo = c_lo[k];
      hi = c_hi[k];
    } else {
      c = __ldcg(&in.id[b + k]);
      lo = __ldcg(&in.lo[b + k]);
      hi = __ldcg(&in.hi[b + k]);
    }
  };
  // this thread's chunk [k0, k1); an odd length keeps a warp's strided
  // shared-memory reads free of bank conflicts
  const int per = ((m + 255) / 256) | 1;
  const int k0 = min(t * per, m), k1 = min(k0 + per, m);
  // centroid bounds of the segment
  {
    float v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int k = k0; k < k1; ++k) {
      int c;
      float4 lo, hi;
      fetch(k, c, lo, hi);
      const float cc[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
      for (int a = 0; a < 3; ++a) {
        v[a] = fminf(v[a], cc[a]);
        v[a + 3] = fmaxf(v[a + 3], cc[a]);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      for (int q = 0; q < 3; ++q) v[q] = fminf(v[q], __shfl_xor_sync(FULL, v[q], o));
      for (int q = 3; q < 6; ++q) v[q] = fmaxf(v[q], __shfl_xor_sync(FULL, v[q], o));
    }
    if (lane == 0 && v[0] <= v[3]) {
      for (int a = 0; a < 3; ++a) {
        atomicMin(&s_cb[a], f2o(v[a]));
        atomicMax(&s_cb[a + 3], f2o(v[a + 3]));
      }
    }
  }
  __syncthreads();
  const float clo[3] = {o2f(s_cb[0]), o2f(s_cb[1]), o2f(s_cb[2])};
  const float cinv[3] = {bin_scale(o2f(s_cb[3]) - clo[0]), bin_scale(o2f(s_cb[4]) - clo[1]),
                         bin_scale(o2f(s_cb[5]) - clo[2])};
  // bin every axis.  A segment of more than kTopSample clusters bins an
  // even subsample of about that many to choose its plane (the partition
  // takes them all).  Lane l of every warp takes samples from the l-th
  // 32nd of the list, so that the lanes of one atomic lie far apart in the
  // list, which keeps neighbouring (same-bin) clusters out of one
  // instruction's lanes; the warps interleave within each lane's part.
  const int sstep = m > kTopSample ? (m + kTopSample - 1) / kTopSample : 1;
  const int n_samp = (m + sstep - 1) / sstep, per_lane = (n_samp + 31) / 32;
  for (int r = w; r < per_lane; r += 8) {
    const int q = lane * per_lane + r;
    if (q >= n_samp) break;
    const int k = q * sstep;
    int c;
    float4 lo, hi;
    fetch(k, c, lo, hi);
    const int b0 = bin_of(0.5f * (lo.x + hi.x), clo[0], cinv[0]);
    const int b1 = bin_of(0.5f * (lo.y + hi.y), clo[1], cinv[1]);
    const int b2 = bin_of(0.5f * (lo.z + hi.z), clo[2], cinv[2]);
    const int n = (int)lo.w;
    const int ilo[3] = {f2o(lo.x), f2o(lo.y), f2o(lo.z)}, ihi[3] = {f2o(hi.x), f2o(hi.y), f2o(hi.z)};
    atomicAdd(&bin_count[0][b0], n);
    atomicAdd(&bin_count[1][b1], n);
    atomicAdd(&bin_count[2][b2], n);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      atomicMin(&bin_lo[0][b0][q], ilo[q]);
      atomicMax(&bin_hi[0][b0][q], ihi[q]);
      atomicMin(&bin_lo[1][b1][q], ilo[q]);
      atomicMax(&bin_hi[1][b1][q], ihi[q]);
      atomicMin(&bin_lo[2][b2][q], ilo[q]);
      atomicMax(&bin_hi[2][b2][q], ihi[q]);
    }
  }
  __syncthreads();
  // the cheapest split plane; by position (ax < 0) when none has a finite
  // cost or the level is deep
  const int best = best_plane(bin_count, bin_lo, bin_hi, s_bc, s_bk);
  const int ax = (best < 0 || level >= kTopForceMedian) ? -1 : best / (kTopBins - 1);
  const int sb = ax < 0 ? 0 : best % (kTopBins - 1);
  // right side (1) or left (0) of position k; by position: the halves in order
  bool by_position = ax < 0;
  const float alo = ax == 0 ? clo[0] : (ax == 1 ? clo[1] : clo[2]);
  const float ainv = ax == 0 ? cinv[0] : (ax == 1 ? cinv[1] : cinv[2]);
  auto side_of = [&](int k, float4 lo, float4 hi) {
    if (by_position) return k >= m / 2 ? 1 : 0;
    const float cl = ax == 0 ? lo.x : (ax == 1 ? lo.y : lo.z);
    const float ch = ax == 0 ? hi.x : (ax == 1 ? hi.y : hi.z);
    return bin_of(0.5f * (cl + ch), alo, ainv) <= sb ? 0 : 1;
  };
  int nleft = 0, before_l = 0, before_r = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    float bx[2][6];
#pragma unroll
    for (int sd = 0; sd < 2; ++sd)
#pragma unroll
      for (int q = 0; q < 6; ++q) bx[sd][q] = q < 3 ? INFINITY : -INFINITY;
    int nl = 0, nr = 0;
    for (int k = k0; k < k1; ++k) {
      int c;
      float4 lo, hi;
      fetch(k, c, lo, hi);
      const int sd = side_of(k, lo, hi);
      if (cached) c_side[k] = (unsigned char)sd;
      nl += sd == 0;
      nr += sd;
      const float v[6] = {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z};
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const float x = sd ? bx[1][q] : bx[0][q];
        const float y = q < 3 ? fminf(x, v[q]) : fmaxf(x, v[q]);
        if (sd) bx[1][q] = y;
        else bx[0][q] = y;
      }
    }
    // exclusive scan of the two counts over the block
    int il = nl, ir = nr;
    for (int o = 1; o < 32; o <<= 1) {
      const int xl = __shfl_up_sync(FULL, il, o), xr = __shfl_up_sync(FULL, ir, o);
      if (lane >= o) {
        il += xl;
        ir += xr;
      }
    }
    if (lane == 31) {
      s_wl[w] = il;
      s_wr[w] = ir;
    }
    __syncthreads();
    int total_l = 0;
    before_l = il - nl;
    before_r = ir - nr;
    for (int q = 0; q < 8; ++q) {
      if (q < w) {
        before_l += s_wl[q];
        before_r += s_wr[q];
      }
      total_l += s_wl[q];
    }
    __syncthreads();   // s_wl / s_wr are read before a second attempt writes them
    if (!by_position && (total_l == 0 || total_l == m)) {
      // not reachable with a finite SAH cost; keep a valid split at the middle
      by_position = true;
      continue;
    }
    nleft = total_l;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
#pragma unroll
        for (int q = 0; q < 3; ++q) bx[sd][q] = fminf(bx[sd][q], __shfl_xor_sync(FULL, bx[sd][q], o));
#pragma unroll
        for (int q = 3; q < 6; ++q) bx[sd][q] = fmaxf(bx[sd][q], __shfl_xor_sync(FULL, bx[sd][q], o));
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int sd = 0; sd < 2; ++sd)
        if (bx[sd][0] <= bx[sd][3])
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            atomicMin(&s_box[sd][q], f2o(bx[sd][q]));
            atomicMax(&s_box[sd][q + 3], f2o(bx[sd][q + 3]));
          }
    }
    break;
  }
  // stable partition: left side ascending from b, right side from b + nleft.
  // A cached segment is ordered in shared memory first (the cache slot of
  // every new position) and copied out with coalesced stores (the chunks'
  // lanes would scatter their stores).
  {
    int pl = before_l, pr = nleft + before_r;
    for (int k = k0; k < k1; ++k) {
      if (cached) {
        const int p = c_side[k] ? pr++ : pl++;
        c_part[p] = k;
      } else {
        int c;
        float4 lo, hi;
        fetch(k, c, lo, hi);
        const int p = b + (side_of(k, lo, hi) ? pr++ : pl++);
        out.id[p] = c;
        out.lo[p] = lo;
        out.hi[p] = hi;
      }
    }
  }
  __syncthreads();
  if (cached) {
    for (int p = t; p < m; p += 256) {
      const int k = c_part[p];
      out.id[b + p] = c_id[k];
      out.lo[b + p] = c_lo[k];
      out.hi[b + p] = c_hi[k];
    }
    __syncthreads();
  }
  for (int sd = 0; sd < 2; ++sd) {
    side_lo[sd] = make_float4(o2f(s_box[sd][0]), o2f(s_box[sd][1]), o2f(s_box[sd][2]), 0.f);
    side_hi[sd] = make_float4(o2f(s_box[sd][3]), o2f(s_box[sd][4]), o2f(s_box[sd][5]), 0.f);
  }
  return nleft;
}

// One block (256 threads) per active segment of this level: binned SAH
// split (16 bins per axis, cost A_L N_L + A_R N_R with N in primitives),
// stable partition of the cluster ids, then the two children are emitted:
// a single cluster becomes a direct link, anything larger a new top node
// (and a segment of the next level).
// seg_in and the input list were written by the previous level (possibly
// by other blocks of the same launch): they are read through L2 (__ldcg).
__device__ __forceinline__ void top_level_body(int level, int top_base, const int* seg_count, const int4* seg_in,
                                               int4* seg_out, int* seg_count_out, CluList in, CluList out,
                                               const int* __restrict__ clu_link, int* top_count, float4* nodes,
                                               BuildInfo* info, int4* small_seg, int* small_count, int cache_cap) {
  // level 0 is one segment over every cluster, which becomes top node 0
  const int nseg = level == 0 ? 1 : __ldcg(&seg_count[level]);
  int t = threadIdx.x;
  if (level == 0 && blockIdx.x == 0 && t == 0) {
    top_count[0] = 1;
    info->height = 1;
  }
  for (int sidx = blockIdx.x; sidx < nseg; sidx += gridDim.x) {
    const int4 sg = level == 0 ? make_int4(0, __ldcg(&seg_count[kTopMaxLevels + 1]), -1, 0) : __ldcg(&seg_in[sidx]);
    int b = sg.x, e = sg.y, node = sg.w;
    int m = e - b;
    float4 slo[2], shi[2];
    int nleft;
    if (m <= 256) {
      nleft = split_small(level, b, e, in, out, slo, shi);
    } else {
      nleft = split_large(level, b, e, in, out, cache_cap, slo, shi);
    }
    if (t < 2) {
      int cb = t == 0 ? b : b + nleft;
      int ce = t == 0 ? b + nleft : e;
      float4 lo = t == 0 ? slo[0] : slo[1], hi = t == 0 ? shi[0] : shi[1];
      int link;
      if (ce - cb == 1) {
        const int c = __ldcg(&out.id[cb]);
        const float h = __ldcg(&out.hi[cb]).w;
        link = clu_link[c];
        // internal nodes on this path: the top levels 0..level, then the cluster's
        atomicMax(&info->height, level + 1 + __float_as_int(h));
      } else {
        // the node id and the queue slot, two independent atomics in flight together
        const bool small = ce - cb <= kTopWarpSeg;
        const int child = atomicAdd(top_count, 1);
        const int slot = atomicAdd(small ? small_count : seg_count_out, 1);
        link = top_base + child;
        if (small) {
          small_seg[slot] = make_int4(cb, ce, child, level + 1);
        } else {
          seg_out[slot] = make_int4(cb, ce, node, child);
        }
        atomicMax(&info->height, level + 2);
      }
      write_child(nodes, top_base + node, t, lo, hi, link);
    }
    __syncthreads();
  }
}

// One warp finishes the subtree of a segment of 2..32 clusters, one cluster
// a lane, all in registers.  Every round splits all unfinished segments of
// the warp at once (their lanes are contiguous): per axis, the clusters are
// ranked by centroid inside their segment, prefix and suffix boxes and
// primitive counts of that order are scanned, and the cheapest split (SAH:
// A_L N_L + A_R N_R over every position, not binned; ties to the lower axis
// and position) is taken; then the lanes are permuted into the two halves.
__device__ __forceinline__ float box_area7(const float* v) {
  float dx = v[3] - v[0], dy = v[4] - v[1], dz = v[5] - v[2];
  if (!(dx >= 0.f) || !(dy >= 0.f) || !(dz >= 0.f)) return 0.f;
  return 2.f * (dx * dy + dy * dz + dz * dx);
}

__device__ __forceinline__ float combine7(int q, float a, float b) {
  return q < 3 ? fminf(a, b) : (q < 6 ? fmaxf(a, b) : a + b);
}

__device__ void build_small_subtree(int4 item, int top_base, CluList in, const int* __restrict__ clu_link,
                                    int* top_count, float4* nodes, BuildInfo* info, int* s_idx, int* s_c,
                                    float4* s_lo, float4* s_hi) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int m = item.y - item.x;
  const bool own = lane < m;
  int c = own ? __ldcg(&in.id[item.x + lane]) : 0;
  float4 lo = own ? __ldcg(&in.lo[item.x + lane]) : make_float4(0.f, 0.f, 0.f, 0.f);
  float4 hi = own ? __ldcg(&in.hi[item.x + lane]) : make_float4(0.f, 0.f, 0.f, 0.f);
  // this lane's segment [sb, se) of lanes; lanes without a cluster are finished singletons
  int sb = own ? 0 : lane, se = own ? m : lane + 1;
  int node = item.z, level = item.w;
  // The subtree has m - 1 inner nodes.  All but its root (allocated by the
  // level that made the segment) come from one block of consecutive ids,
  // reserved with one atomic, in breadth-first order.
  int sub_base = 0, sub_next = 0;
  if (lane == 0 && m > 2) sub_base = atomicAdd(top_count, m - 2);
  sub_base = __shfl_sync(FULL, sub_base, 0);
  for (int round = 0; round < 32; ++round) {
    const bool act = se - sb >= 2;
    if (!__any_sync(FULL, act)) break;
    const float cen[3] = {0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z)};
    // The three axes advance together, so that a lone warp has three
    // independent shuffle chains in flight.  The lanes' segments differ, so
    // every test below is written without short-circuit operators: a branch
    // on them would diverge.
    const unsigned seg_w = (unsigned)(se - sb);
    int rank[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const bool in = (unsigned)(j - sb) < seg_w;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float cj = __shfl_sync(FULL, cen[a], j);
        rank[a] += (int)(in & ((cj < cen[a]) | ((cj == cen[a]) & (j < lane))));
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) s_idx[32 * a + sb + rank[a]] = lane;
    __syncwarp();
    int src[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) src[a] = s_idx[32 * a + lane];
    __syncwarp();
    // per axis, boxes and primitive counts of the prefixes and suffixes of
    // the segment's clusters in that axis' order
    const float v[7] = {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z, lo.w};
    float pre[3][7], suf[3][7], right[3][7];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int q = 0; q < 7; ++q) pre[a][q] = suf[a][q] = __shfl_sync(FULL, v[q], src[a]);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const bool up = lane - o >= sb, down = lane + o < se;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int q = 0; q < 7; ++q) {
          const float x = __shfl_up_sync(FULL, pre[a][q], o);
          const float y = __shfl_down_sync(FULL, suf[a][q], o);
          pre[a][q] = up ? combine7(q, pre[a][q], x) : pre[a][q];
          suf[a][q] = down ? combine7(q, suf[a][q], y) : suf[a][q];
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int q = 0; q < 7; ++q) right[a][q] = __shfl_down_sync(FULL, suf[a][q], 1);   // suffix from the next position
    // SAH of the split after each position; per axis the cheapest in the
    // segment, ties to the lower position
    const bool valid = act & (lane + 1 < se);
    float cost[3];
    int pos[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cost[a] = valid ? box_area7(pre[a]) * pre[a][6] + box_area7(right[a]) * right[a][6] : INFINITY;
      pos[a] = lane;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const bool up = lane - o >= sb;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float oc = __shfl_up_sync(FULL, cost[a], o);
        const int op = __shfl_up_sync(FULL, pos[a], o);
        const bool take = up & ((oc < cost[a]) | ((oc == cost[a]) & (op < pos[a])));
        cost[a] = take ? oc : cost[a];
        pos[a] = take ? op : pos[a];
      }
    }
    // the cheapest axis, ties to the lower axis
    float best = INFINITY;
    int best_ax = 0, best_k = -1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float seg_cost = __shfl_sync(FULL, cost[a], se - 1);
      const int seg_pos = __shfl_sync(FULL, pos[a], se - 1);
      const bool better = seg_cost < best;
      best = better ? seg_cost : best;
      best_ax = better ? a : best_ax;
      best_k = better ? seg_pos : best_k;
    }
    // the two children's boxes: the chosen axis' prefix at best_k and the
    // suffix after it (the source lane is in this segment, so it chose the
    // same axis)
    const int from = best_k < 0 ? lane : best_k;
    float bl[7], br[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      const float p = best_ax == 0 ? pre[0][q] : (best_ax == 1 ? pre[1][q] : pre[2][q]);
      const float r = best_ax == 0 ? right[0][q] : (best_ax == 1 ? right[1][q] : right[2][q]);
      bl[q] = __shfl_sync(FULL, p, from);
      br[q] = __shfl_sync(FULL, r, from);
    }
    if (act && best_k < 0) {
      // no finite cost (not reachable for finite boxes): halves of the x
      // order under boxes that every ray enters
      best_ax = 0;
      best_k = sb + (se - sb) / 2 - 1;
      for (int q = 0; q < 7; ++q) bl[q] = br[q] = q < 3 ? -INFINITY : INFINITY;
    }
    // the lanes in the chosen order: left child [sb, best_k], right child [best_k + 1, se)
    const int dst = act ? sb + (best_ax == 0 ? rank[0] : best_ax == 1 ? rank[1] : rank[2]) : lane;
    s_c[dst] = c;
    s_lo[dst] = lo;
    s_hi[dst] = hi;
    __syncwarp();
    c = s_c[lane];
    lo = s_lo[lane];
    hi = s_hi[lane];
    __syncwarp();
    const int k = act ? best_k : lane;
    const int c_right = __shfl_sync(FULL, c, min(k + 1, 31));
    const float h_right = __shfl_sync(FULL, hi.w, min(k + 1, 31));   // the right cluster's height
    // this round's new nodes, numbered in lane order (left before right)
    // after those of the earlier rounds
    const bool lead = act && lane == sb;
    const bool new_l = lead && k + 1 - sb > 1, new_r = lead && se - (k + 1) > 1;
    const unsigned ml = __ballot_sync(FULL, new_l), mr = __ballot_sync(FULL, new_r);
    const unsigned below = (1u << lane) - 1u;
    const int id_l = sub_base + sub_next + __popc(ml & below) + __popc(mr & below);
    sub_next += __popc(ml) + __popc(mr);
    int cnode_l = -1, cnode_r = -1;
    if (lead) {
      int link_l, link_r;
      if (!new_l) {
        link_l = clu_link[c];
        atomicMax(&info->height, level + 1 + __float_as_int(hi.w));
      } else {
        cnode_l = id_l;
        link_l = top_base + cnode_l;
        atomicMax(&info->height, level + 2);
      }
      if (!new_r) {
        link_r = clu_link[c_right];
        atomicMax(&info->height, level + 1 + __float_as_int(h_right));
      } else {
        cnode_r = id_l + (new_l ? 1 : 0);
        link_r = top_base + cnode_r;
        atomicMax(&info->height, level + 2);
      }
      write_child(nodes, top_base + node, 0, make_float4(bl[0], bl[1], bl[2], 0.f),
                  make_float4(bl[3], bl[4], bl[5], 0.f), link_l);
      write_child(nodes, top_base + node, 1, make_float4(br[0], br[1], br[2], 0.f),
                  make_float4(br[3], br[4], br[5], 0.f), link_r);
    }
    cnode_l = __shfl_sync(FULL, cnode_l, sb);
    cnode_r = __shfl_sync(FULL, cnode_r, sb);
    if (act) {
      if (lane <= k) {
        se = k + 1;
        node = cnode_l;
      } else {
        sb = k + 1;
        node = cnode_r;
      }
      ++level;
    }
  }
}

// Every small segment of the top-level rebuild, one warp each.  Segment i
// goes to warp i / gridDim of block i % gridDim, so that the segments
// spread over all SMs (a warp's rounds are latency bound) before any block
// takes a second one.
__device__ __forceinline__ void top_small_body(const int* seg_count, const int4* small_seg, int top_base, CluList la,
                                               CluList lb, const int* __restrict__ clu_link, int* top_count,
                                               float4* nodes, BuildInfo* info) {
  __shared__ int s_idx[8][3 * 32], s_c[8][32];
  __shared__ float4 s_lo[8][32], s_hi[8][32];
  const int w = threadIdx.x >> 5;
  const int n_small = __ldcg(&seg_count[kTopMaxLevels + 2]);
  const int warps = (int)(gridDim.x * (blockDim.x >> 5));
  for (int i = w * (int)gridDim.x + (int)blockIdx.x; i < n_small; i += warps) {
    int4 item = __ldcg(&small_seg[i]);
    // a level-L segment is in the buffer its parent's split wrote
    build_small_subtree(item, top_base, (item.w & 1) ? lb : la, clu_link, top_count, nodes, info, s_idx[w], s_c[w],
                        s_lo[w], s_hi[w]);
  }
}

__global__ void __launch_bounds__(256) k_top_small(const int* seg_count, const int4* small_seg, int top_base,
                                                   CluList la, CluList lb, const int* __restrict__ clu_link,
                                                   int* top_count, float4* nodes, BuildInfo* info) {
  top_small_body(seg_count, small_seg, top_base, la, lb, clu_link, top_count, nodes, info);
}

__global__ void __launch_bounds__(256) k_top_level(int level, int top_base, const int* seg_count, const int4* seg_in,
                                                   int4* seg_out, int* seg_count_out, CluList in, CluList out,
                                                   const int* __restrict__ clu_link, int* top_count, float4* nodes,
                                                   BuildInfo* info, int4* small_seg, int* small_count,
                                                   int cache_cap) {
  top_level_body(level, top_base, seg_count, seg_in, seg_out, seg_count_out, in, out, clu_link, top_count, nodes, info,
                 small_seg, small_count, cache_cap);
}

// Every level in one cooperative launch: the blocks meet at a grid-wide
// barrier between levels and stop at the first level without segments.
__global__ void __launch_bounds__(256) k_top_all(int top_base, int* seg_count, int4* seg_a, int4* seg_b, CluList la,
                                                 CluList lb, const int* __restrict__ clu_link, int* top_count,
                                                 float4* nodes, BuildInfo* info, int4* small_seg, int cache_cap) {
  cg::grid_group grid = cg::this_grid();
  for (int level = 0; level < kTopMaxLevels; ++level) {
    if (level > 0 && __ldcg(&seg_count[level]) == 0) break;   // the same value in every block after the barrier
    bool odd = level & 1;
    top_level_body(level, top_base, seg_count, odd ? seg_b : seg_a, odd ? seg_a : seg_b, seg_count + level + 1,
                   odd ? lb : la, odd ? la : lb, clu_link, top_count, nodes, info, small_seg,
                   seg_count + kTopMaxLevels + 2, cache_cap);
    grid.sync();
  }
  // the small segments, one warp each, with no more barriers
  top_small_body(seg_count, small_seg, top_base, la, lb, clu_link, top_count, nodes, info);
}

// ---------------------------------------------------------------------------
// 8. 4-wide traversal tree.  A 4-wide node stands for one internal node of
//    the binary tree and takes its children; while it has fewer than four,
//    the internal child with the largest surface area is replaced by its
//    own two children.  What a 4-wide node holds depends on its binary
//    node's subtree alone, so every binary node gets its 4-wide node at its
//    own index, in parallel: a child slot that is an internal binary node
//    links to that node's 4-wide node.  Walking from the root reaches
//    exactly the nodes a top-down collapse would make; the others are never
//    visited.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bin_child(const float4* __restrict__ bin, int node, int c, float* lo, float* hi,
                                          int& link) {
  const float4* n = bin + 4 * (size_t)node;
  float4 xy = __ldg(n + c), z = __ldg(n + 2), l = __ldg(n + 3);
  lo[0] = xy.x;
  hi[0] = xy.y;
  lo[1] = xy.z;
  hi[1] = xy.w;
  lo[2] = c == 0 ? z.x : z.z;
  hi[2] = c == 0 ? z.y : z.w;
  link = __float_as_int(c == 0 ? l.x : l.y);
}

__device__ __forceinline__ float half_area(const float* lo, const float* hi) {
  float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
  return dx * dy + dy * dz + dz * dx;
}

// Slots x0 .. x1 - 1.  Slots past the LBVH's n_lbvh internal nodes are top
// nodes; only the first *top_count of them exist (none without a top
// rebuild: top_count NULL, which a launch over LBVH slots alone passes too).
__global__ void __launch_bounds__(256) k_collapse4(const float4* __restrict__ bin, int x0, int x1, int n_bin,
                                                   int n_lbvh, const int* __restrict__ top_count,
                                                   const int* __restrict__ n_clusters, BuildInfo* info, int top_base,
                                                   float4* __restrict__ out) {
  const int x = x0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (x == x0 && top_count) {
    // the rebuilt top's counts and root, for rt_bvh_get_info
    info->n_top = *top_count;
    info->n_clusters = *n_clusters;
    info->root = top_base;
  }
  if (x >= x1) return;
  if (x >= n_lbvh && (top_count == nullptr || x - n_lbvh >= __ldg(top_count))) return;   // an unused slot
  // Slots are indexed only by constants once the loops unroll, so they stay
  // in registers; the slot chosen at run time is written through selects.
  float lo[4][3], hi[4][3];
  int link[4] = {kEmptyLink, kEmptyLink, kEmptyLink, kEmptyLink};
  int ns = 2;
  bin_child(bin, x, 0, lo[0], hi[0], link[0]);
  bin_child(bin, x, 1, lo[1], hi[1], link[1]);
#pragma unroll
  for (int m = 2; m < 4; ++m) {
    // the inner child of largest area (the first on ties) is opened
    int best = -1;
    float ba = -1.f;
#pragma unroll
    for (int k = 0; k < m; ++k) {
      const bool inner = link[k] >= 0 && link[k] < n_bin;   // a leaf stays a leaf
      const float a = inner ? half_area(lo[k], hi[k]) : -1.f;
      const bool take = inner && a > ba;
      ba = take ? a : ba;
      best = take ? k : best;
    }
    if (best < 0) break;
    int c = link[0];
#pragma unroll
    for (int k = 1; k < m; ++k) c = best == k ? link[k] : c;
    float l0[3], h0[3];
    int c0;
    bin_child(bin, c, 1, lo[m], hi[m], link[m]);
    bin_child(bin, c, 0, l0, h0, c0);
#pragma unroll
    for (int k = 0; k < m; ++k) {
      const bool here = best == k;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        lo[k][a] = here ? l0[a] : lo[k][a];
        hi[k][a] = here ? h0[a] : hi[k][a];
      }
      link[k] = here ? c0 : link[k];
    }
    ns = m + 1;
  }
  float r[6][4];
  int out_link[4];
  for (int k = 0; k < 4; ++k) {
    bool used = k < ns;
    out_link[k] = used ? link[k] : kEmptyLink;
    for (int a = 0; a < 3; ++a) {
      r[2 * a][k] = used ? lo[k][a] : INFINITY;
      r[2 * a + 1][k] = used ? hi[k][a] : -INFINITY;
    }
  }
  float4* o = out + 8 * (size_t)x;
  for (int q = 0; q < 6; ++q) o[q] = make_float4(r[q][0], r[q][1], r[q][2], r[q][3]);
  o[6] = make_float4(__int_as_float(out_link[0]), __int_as_float(out_link[1]), __int_as_float(out_link[2]),
                     __int_as_float(out_link[3]));
  o[7] = make_float4(__int_as_float(ns), 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------------------
// 7. traversal layout of the LBVH nodes
// ---------------------------------------------------------------------------
__global__ void k_layout(int n, const int* __restrict__ lch, const int* __restrict__ rch, const int2* __restrict__ range,
                         const float4* __restrict__ node_lo, const float4* __restrict__ node_hi,
                         const unsigned* __restrict__ vals, const float4* __restrict__ aabb_lo,
                         const float4* __restrict__ aabb_hi, float4* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  float4 lo[2], hi[2];
  int link[2];
  int kids[2] = {lch[i], rch[i]};
  for (int k = 0; k < 2; ++k) {
    int c = kids[k];
    if (c < 0) {
      unsigned pid = vals[~c];
      lo[k] = aabb_lo[pid];
      hi[k] = aabb_hi[pid];
      link[k] = leaf_link(~c, 1);
    } else {
      lo[k] = node_lo[c];
      hi[k] = node_hi[c];
      int meta = __float_as_int(hi[k].w);
      if ((meta >> 8) & 1) {
        int2 rg = range[c];
        link[k] = leaf_link(rg.x, rg.y - rg.x + 1);
      } else {
        link[k] = c;
      }
    }
  }
  float4* o = out + 4 * (size_t)i;
  o[0] = make_float4(lo[0].x, hi[0].x, lo[0].y, hi[0].y);
  o[1] = make_float4(lo[1].x, hi[1].x, lo[1].y, hi[1].y);
  o[2] = make_float4(lo[0].z, hi[0].z, lo[1].z, hi[1].z);
  o[3] = make_float4(__int_as_float(link[0]), __int_as_float(link[1]), 0.f, 0.f);
}

// one primitive, 4-wide: a root with one used slot
__global__ void k_wide_single(const float4* __restrict__ aabb_lo, const float4* __restrict__ aabb_hi,
                              float4* __restrict__ out) {
  float4 lo = aabb_lo[0], hi = aabb_hi[0];
  out[0] = make_float4(lo.x, INFINITY, INFINITY, INFINITY);
  out[1] = make_float4(hi.x, -INFINITY, -INFINITY, -INFINITY);
  out[2] = make_float4(lo.y, INFINITY, INFINITY, INFINITY);
  out[3] = make_float4(hi.y, -INFINITY, -INFINITY, -INFINITY);
  out[4] = make_float4(lo.z, INFINITY, INFINITY, INFINITY);
  out[5] = make_float4(hi.z, -INFINITY, -INFINITY, -INFINITY);
  out[6] = make_float4(__int_as_float(leaf_link(0, 1)), __int_as_float(kEmptyLink), __int_as_float(kEmptyLink),
                       __int_as_float(kEmptyLink));
  out[7] = make_float4(__int_as_float(1), 0.f, 0.f, 0.f);
}

// one primitive: a root whose second child box is empty
__global__ void k_layout_single(const float4* __restrict__ aabb_lo, const float4* __restrict__ aabb_hi,
                                float4* __restrict__ out, BuildInfo* info, int* __restrict__ cb) {
  for (int t = 0; t < 6; ++t) reset_bounds(cb, t);
  float4 lo = aabb_lo[0], hi = aabb_hi[0];
  out[0] = make_float4(lo.x, hi.x, lo.y, hi.y);
  out[1] = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
  out[2] = make_float4(lo.z, hi.z, INFINITY, -INFINITY);
  out[3] = make_float4(__int_as_float(leaf_link(0, 1)), __int_as_float(leaf_link(0, 1)), 0.f, 0.f);
  info->height = 1;
  info->sah = kCostTrav + kCostIsect;
  info->sah_lbvh = info->sah;
  info->root = 0;
  info->n_clusters = 0;
  info->n_top = 0;
  info->max_leaf = 1;
}

__global__ void k_gather_prims(const unsigned* __restrict__ vals, int n, const float4* __restrict__ in,
                               float4* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  int p = i / 3, r = i - 3 * p;
  unsigned v = min(vals[p], (unsigned)(n - 1));
  out[i] = in[3 * (size_t)v + r];
}

__global__ void k_info_lbvh(const float4* __restrict__ node_lo, const float4* __restrict__ node_hi,
                            const float* __restrict__ cost_lbvh, BuildInfo* info, int root) {
  info->height = __float_as_int(node_hi[0].w) & 0xff;
  info->sah = node_lo[0].w;
  info->sah_lbvh = cost_lbvh[0];
  info->root = root;
  info->n_clusters = 0;
  info->n_top = 0;
  info->max_leaf = kMaxLeaf;
}

}  // namespace rtb

using namespace rtb;

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
namespace rtb {

static rt_status carve(rt_scene* s, int n, BuildScratch& b) {
  size_t tiles = (size_t)(n + kSortTile - 1) / kSortTile;
  size_t hist_n = 256 * std::max(tiles, (size_t)kSortCoopMaxBlocks);   // per-tile or per-block digit counts
  size_t parts = std::max((hist_n + kScanBlock - 1) / kScanBlock + 1, (size_t)256);   // scan partials / digit totals
  size_t N = (size_t)std::max(n, 2);
  size_t off = 0;
  size_t sz[48];
  int k = 0;
  sz[k++] = N * 16;  // aabb_lo
  sz[k++] = N * 16;  // aabb_hi
  sz[k++] = N * 4;   // keys0
  sz[k++] = N * 4;   // vals0
  sz[k++] = N * 4;   // keys1
  sz[k++] = N * 4;   // vals1
  sz[k++] = hist_n * 4 + 16;
  sz[k++] = parts * 4 + 16;
  sz[k++] = N * 4;   // lch
  sz[k++] = N * 4;   // rch
  sz[k++] = N * 4;   // parent
  sz[k++] = N * 4;   // leaf_parent
  sz[k++] = N * 4;   // flags
  sz[k++] = N * 8;   // range
  sz[k++] = N * 16;  // node_lo
  sz[k++] = N * 16;  // node_hi
  sz[k++] = N * 4;   // cost_lbvh
  sz[k++] = 64;      // cent_bounds
  sz[k++] = N * 4;   // clu_a
  sz[k++] = N * 4;   // clu_b
  sz[k++] = N * 4;   // clu_link
  sz[k++] = N * 16;  // clu_lo
  sz[k++] = N * 16;  // clu_hi
  sz[k++] = N * 16;  // clu_lo_b
  sz[k++] = N * 16;  // clu_hi_b
  sz[k++] = N * 16;  // seg_a
  sz[k++] = N * 16;  // seg_b
  sz[k++] = (kTopMaxLevels + 3) * 4;   // seg_count: levels, n_clusters, small segments
  sz[k++] = 16;      // top_count
  sz[k++] = N * 16;  // small_seg
  sz[k++] = sizeof(BuildInfo);
  static_assert(sizeof(sz) / sizeof(sz[0]) >= 36, "scratch region table too small");
  size_t total = 0;
  for (int i = 0; i < k; ++i) total += align_up(sz[i]);
  rt_status st = ensure(s->build_tmp, total);
  if (st) return st;
  char* base = (char*)s->build_tmp.p;
  void* ptr[48];
  for (int i = 0; i < k; ++i) {
    ptr[i] = base + off;
    off += align_up(sz[i]);
  }
  int q = 0;
  b.aabb_lo = (float4*)ptr[q++];
  b.aabb_hi = (float4*)ptr[q++];
  b.keys0 = (unsigned*)ptr[q++];
  b.vals0 = (unsigned*)ptr[q++];
  b.keys1 = (unsigned*)ptr[q++];
  b.vals1 = (unsigned*)ptr[q++];
  b.hist = (unsigned*)ptr[q++];
  b.partials = (unsigned*)ptr[q++];
  b.lch = (int*)ptr[q++];
  b.rch = (int*)ptr[q++];
  b.parent = (int*)ptr[q++];
  b.leaf_parent = (int*)ptr[q++];
  b.flags = (int*)ptr[q++];
  b.range = (int2*)ptr[q++];
  b.node_lo = (float4*)ptr[q++];
  b.node_hi = (float4*)ptr[q++];
  b.cost_lbvh = (float*)ptr[q++];
  b.cent_bounds = (int*)ptr[q++];
  b.clu_a = (int*)ptr[q++];
  b.clu_b = (int*)ptr[q++];
  b.clu_link = (int*)ptr[q++];
  b.clu_lo = (float4*)ptr[q++];
  b.clu_hi = (float4*)ptr[q++];
  b.clu_lo_b = (float4*)ptr[q++];
  b.clu_hi_b = (float4*)ptr[q++];
  b.seg_a = (int4*)ptr[q++];
  b.seg_b = (int4*)ptr[q++];
  b.seg_count = (int*)ptr[q++];
  b.top_count = (int*)ptr[q++];
  b.small_seg = (int4*)ptr[q++];
  b.info = (BuildInfo*)ptr[q++];
  return RT_OK;
}

// Cluster size of the top-level rebuild: aims at a few thousand clusters.
static int cluster_max_for(int n) {
  int c = 64;
  while ((int64_t)n / c > 16384) c *= 2;
  return c;
}

// The 4-wide traversal tree: one 4-wide node per binary node slot, at the
// same index (the root is the binary root), for slots x0 .. x1 - 1.  The
// top's counts are recorded by the launch that takes slot n - 1, the first
// top node, when there is a top (top_base >= 0).
static rt_status collapse4(rt_scene* s, const BuildScratch& b, const float4* nodes, int n_bin, int top_base,
                           int x0, int x1, cudaStream_t st) {
  rt_status rs = ensure(s->nodes4, (size_t)n_bin * 128);
  if (rs) return rs;
  s->n_nodes4 = n_bin;
  if (s->n_prims == 1) {
    k_wide_single<<<1, 1, 0, st>>>(b.aabb_lo, b.aabb_hi, (float4*)s->nodes4.p);
  } else if (x1 > x0) {
    const int n_lbvh = (int)s->n_prims - 1;
    const bool counts = top_base >= 0 && x0 <= n_lbvh && n_lbvh < x1;
    k_collapse4<<<(x1 - x0 + 255) / 256, 256, 0, st>>>(nodes, x0, x1, n_bin, n_lbvh, counts ? b.top_count : nullptr,
                                                       b.seg_count + kTopMaxLevels + 1, b.info, top_base,
                                                       (float4*)s->nodes4.p);
  }
  return cuda_error(cudaGetLastError(), "rt_bvh_build: 4-wide tree");
}

static rt_status ensure_build_side(rt_scene* s) {
  if (s->ev_build_join) return RT_OK;
  rt_status rs = ensure_side_stream(s);
  if (rs) return rs;
  cudaError_t e = cudaEventCreateWithFlags(&s->ev_build_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_build_join, cudaEventDisableTiming);
  return cuda_error(e, "rt_bvh_build: side stream");
}

static rt_status bvh_build_launch(rt_scene* s, cudaStream_t st);

// The buffers a build's launches name, by their allocation generations.
static void build_key(const rt_scene* s, unsigned key[6]) {
  key[0] = (unsigned)s->n_prims;
  key[1] = s->build_tmp.gen;
  key[2] = s->nodes.gen;
  key[3] = s->nodes4.gen;
  key[4] = s->prims_id.gen;
  key[5] = s->prims_leaf.gen;
}

// A build: its ~20 launches (kernels, memsets, the side stream's fork and
// join) depend only on the scene's size and buffers.  A build that found
// the buffers unchanged by the build before it captures its launches into
// a CUDA graph, and later builds with the same buffers replay that graph
// on their stream (one launch instead of twenty).  A build called on a
// stream that is being captured launches directly, into the caller's graph.
rt_status bvh_build(rt_scene* s, cudaStream_t st) {
  if (s->n_prims < 2) return bvh_build_launch(s, st);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return bvh_build_launch(s, st);
  }
  unsigned key[6];
  build_key(s, key);
  const bool same = memcmp(key, s->build_key, sizeof(key)) == 0;
  if (s->build_exec && same) {
    cudaError_t e = cudaGraphLaunch(s->build_exec, st);
    if (e != cudaSuccess) return cuda_error(e, "rt_bvh_build: graph launch");
    s->root = s->build_root;
    s->lbvh_cut = s->build_lbvh_cut;
    s->n_nodes_total = s->build_nodes_total;
    s->n_nodes4 = s->build_nodes4;
    s->last_build_launches = s->build_launches;
    s->built = true;
    return RT_OK;
  }
  if (s->build_exec) {
    cudaGraphExecDestroy(s->build_exec);
    s->build_exec = nullptr;
  }
  rt_status rs = bvh_build_launch(s, st);
  if (rs) return rs;
  unsigned after[6];
  build_key(s, after);
  if (memcmp(after, key, sizeof(key)) != 0 || s->build_cap_failed) {
    memcpy(s->build_key, after, sizeof(after));   // buffers were (re)allocated: capture next time
    return RT_OK;
  }
  // nothing was allocated: the same launches, captured for the next builds
  cudaError_t e = cudaSuccess;
  if (!s->build_cap) e = cudaStreamCreateWithFlags(&s->build_cap, cudaStreamNonBlocking);
  cudaGraph_t graph = nullptr;
  if (e == cudaSuccess) e = cudaStreamBeginCapture(s->build_cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rs = bvh_build_launch(s, s->build_cap);
    e = cudaStreamEndCapture(s->build_cap, &graph);
    if (rs != RT_OK && e == cudaSuccess) e = cudaErrorUnknown;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&s->build_exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    // no graph then: every build launches directly
    cudaGetLastError();
    s->build_exec = nullptr;
    s->build_cap_failed = true;
    return RT_OK;
  }
  memcpy(s->build_key, key, sizeof(key));
  s->build_root = s->root;
  s->build_lbvh_cut = s->lbvh_cut;
  s->build_nodes_total = s->n_nodes_total;
  s->build_nodes4 = s->n_nodes4;
  s->build_launches = s->last_build_launches;
  return RT_OK;
}

static rt_status bvh_build_launch(rt_scene* s, cudaStream_t st) {
  int n = (int)s->n_prims;
  if (n == 0) {
    s->root = -1;
    s->built = true;
    return RT_OK;
  }
  BuildScratch b;
  rt_status rs = carve(s, n, b);
  if (rs) return rs;
  s->lbvh_cut = 0;
  // nodes: LBVH internal nodes [0, n-1) + top nodes [n-1, 2n-2)
  size_t slots = (size_t)std::max(2 * n, 2);
  if ((rs = ensure(s->nodes, slots * 64))) return rs;
  s->n_nodes_total = (int64_t)slots;
  float4* nodes = (float4*)s->nodes.p;
  int tb = 256, grid = (n + tb - 1) / tb;
  int L = 0;   // launches (kernels + memsets) of this build
  if (s->bounds_gen != s->build_tmp.gen) {
    k_init_bounds<<<1, 32, 0, st>>>(b.cent_bounds);   // fresh scratch
    s->bounds_gen = s->build_tmp.gen;
    L += 1;
  }
  k_prim_bounds<<<grid, tb, 0, st>>>((const float4*)s->prims_id.p, n, b.aabb_lo, b.aabb_hi, b.cent_bounds);
  L += 1;
  if (n == 1) {
    cudaMemsetAsync(b.vals0, 0, 4, st);
    k_layout_single<<<1, 1, 0, st>>>(b.aabb_lo, b.aabb_hi, nodes, b.info, b.cent_bounds);
    k_gather_prims<<<1, 32, 0, st>>>(b.vals0, 1, (const float4*)s->prims_id.p, (float4*)s->prims_leaf.p);
    s->root = 0;
    if ((rs = collapse4(s, b, nodes, (int)slots, -1, 0, (int)slots, st))) return rs;
    s->last_build_launches = L + 4;
    s->built = true;
    return cuda_error(cudaGetLastError(), "rt_bvh_build");
  }
  const int key_bits = morton_key_bits(n);
  const bool odd = sort_passes(key_bits) & 1;
  k_morton<<<grid, tb, 0, st>>>(b.aabb_lo, b.aabb_hi, n, b.cent_bounds, 30 - key_bits, odd ? b.keys1 : b.keys0,
                                odd ? b.vals1 : b.vals0, b.flags, b.parent, b.leaf_parent);
  L += 1 + radix_sort_pairs(s, b, n, key_bits, st);
  static_assert(kTopMaxLevels + 3 <= 256, "k_hierarchy's first block clears the top counters");
  k_hierarchy<<<grid, tb, 0, st>>>(b.keys0, n, b.lch, b.rch, b.parent, b.leaf_parent, b.range, b.cent_bounds,
                                   b.seg_count, kTopMaxLevels + 3);
  int cmax = cluster_max_for(n);
  const bool top = n > 2 * cmax;   // the top levels are rebuilt over clusters of <= cmax primitives
  // clusters of at most kWarpRefitMax primitives are refitted one warp each
  // after they are found (k_refit_clusters); otherwise k_refit climbs first
  const bool warp_refit = top && cmax <= kWarpRefitMax;
  if (!warp_refit)
    k_refit<<<grid, tb, 0, st>>>(n, top ? cmax : n, b.vals0, b.aabb_lo, b.aabb_hi, b.lch, b.rch, b.parent,
                                 b.leaf_parent, b.range, b.node_lo, b.node_hi, b.cost_lbvh, b.flags);
  // the LBVH above the clusters only feeds the plain LBVH's cost, which
  // rt_bvh_get_info computes when asked (upper_refit)
  s->lbvh_cut = top ? cmax : 0;
  // With a top rebuild, the binary layout of the LBVH nodes, the primitives
  // in leaf order and the 4-wide nodes of the LBVH slots do not depend on
  // it: they run on the scene's side stream beside it (forked below, once
  // the clusters are found), on the SMs that its few active blocks leave
  // idle.  (Forked right after k_refit, to overlap the cluster search too,
  // the step was 4 us slower.)
  const bool fork = top && ensure_build_side(s) == RT_OK;
  auto layout = [&](cudaStream_t sl) {
    k_layout<<<grid, tb, 0, sl>>>(n, b.lch, b.rch, b.range, b.node_lo, b.node_hi, b.vals0, b.aabb_lo, b.aabb_hi,
                                  nodes);
    k_gather_prims<<<(3 * n + 255) / 256, 256, 0, sl>>>(b.vals0, n, (const float4*)s->prims_id.p,
                                                        (float4*)s->prims_leaf.p);
  };
  if (!fork) layout(st);
  if (!top) k_info_lbvh<<<1, 1, 0, st>>>(b.node_lo, b.node_hi, b.cost_lbvh, b.info, 0);
  L += top ? 4 : 5;   // k_hierarchy, k_refit, k_layout, k_gather_prims (and k_info_lbvh)
  s->root = 0;
  if (top) {
    // top levels: binned SAH over the Morton clusters
    int top_base = n - 1;
    int* n_clusters_dev = b.seg_count + kTopMaxLevels + 1;
    // (k_hierarchy cleared the counters.)  Every top node the rebuild
    // allocates gets both children written; the slots past them are never
    // read (k_collapse4 stops at *top_count).
    k_find_clusters<<<grid, tb, 0, st>>>(n, cmax, b.lch, b.rch, b.range, b.node_lo, b.node_hi, b.vals0, b.aabb_lo,
                                         b.aabb_hi, n_clusters_dev, b.clu_a, b.clu_link, b.clu_lo, b.clu_hi,
                                         warp_refit ? 1 : 0);
    if (warp_refit) {
      k_refit_clusters<<<8 * s->sm_count, 32 * kWarpRefitWarps, 0, st>>>(
          n, b.vals0, b.aabb_lo, b.aabb_hi, b.lch, b.rch, b.parent, b.leaf_parent, b.range, b.node_lo, b.node_hi,
          b.cost_lbvh, n_clusters_dev, b.clu_link, b.clu_lo, b.clu_hi);
    }
    if (fork) {
      cudaEventRecord(s->ev_build_fork, st);
      cudaStreamWaitEvent(s->side, s->ev_build_fork, 0);
      layout(s->side);
      if ((rs = collapse4(s, b, nodes, (int)slots, n - 1, 0, n - 1, s->side))) return rs;
      cudaEventRecord(s->ev_build_join, s->side);
      L += 1;
    }
    int top_grid = std::max(1, 2 * s->sm_count);
    // dynamic shared memory: the cluster cache of one segment
    int cache_cap = kTopCache;
    const size_t dyn = (size_t)cache_cap * 41;   // per cached cluster: lo, hi, id, partitioned id, side
    static int coop_blocks = -1;
    if (coop_blocks < 0) {
      int coop = 0, per_sm = 0;
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device);
      cudaFuncSetAttribute(k_top_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      cudaFuncSetAttribute(k_top_level, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_top_all, 256, dyn);
      coop_blocks = coop ? std::min(per_sm, 1) * s->sm_count : 0;   // one an SM: cheaper grid barriers
    }
    bool launched = false;
    CluList la{b.clu_a, b.clu_lo, b.clu_hi}, lb{b.clu_b, b.clu_lo_b, b.clu_hi_b};
    if (coop_blocks > 0) {
      int tb_ = top_base;
      void* args[] = {&tb_, &b.seg_count, &b.seg_a, &b.seg_b, &la, &lb, &b.clu_link,
                      &b.top_count, &nodes, &b.info, &b.small_seg, &cache_cap};
      launched = cudaLaunchCooperativeKernel((void*)k_top_all, coop_blocks, 256, args, dyn, st) == cudaSuccess;
      if (!launched) cudaGetLastError();
      L += launched ? 1 - kTopMaxLevels : 0;
    }
    for (int level = 0; !launched && level < kTopMaxLevels; ++level) {
      bool odd = level & 1;
      k_top_level<<<top_grid, 256, dyn, st>>>(level, top_base, b.seg_count, odd ? b.seg_b : b.seg_a,
                                              odd ? b.seg_a : b.seg_b, b.seg_count + level + 1,
                                              odd ? lb : la, odd ? la : lb, b.clu_link, b.top_count, nodes, b.info,
                                              b.small_seg, b.seg_count + kTopMaxLevels + 2, cache_cap);
    }
    if (!launched) {
      k_top_small<<<top_grid, 256, 0, st>>>(b.seg_count, b.small_seg, top_base, la, lb, b.clu_link, b.top_count,
                                            nodes, b.info);
      L += 1;
    }
    L += 1 + kTopMaxLevels;   // k_collapse4 records the top's counts and root
    s->root = top_base;
  }
  if (fork) {
    cudaStreamWaitEvent(st, s->ev_build_join, 0);
    rs = collapse4(s, b, nodes, (int)slots, s->root, n - 1, (int)slots, st);
  } else {
    rs = collapse4(s, b, nodes, (int)slots, top ? s->root : -1, 0, (int)slots, st);
  }
  if (rs) return rs;
  L += 1;
  s->last_build_launches = L;
  s->built = true;
  return cuda_error(cudaGetLastError(), "rt_bvh_build");
}

}  // namespace rtb

extern "C" {

rt_status rt_bvh_build(rt_scene* s, void* stream) {
  if (!s) return set_error(RT_ERR_INVALID_ARG, "rt_bvh_build: scene is NULL");
  return bvh_build(s, (cudaStream_t)stream);
}

rt_status rt_bvh_get_info(rt_scene* s, rt_bvh_info* info, void* stream) {
  if (!s || !info) return set_error(RT_ERR_INVALID_ARG, "rt_bvh_get_info: NULL argument");
  if (!s->built) return set_error(RT_ERR_NOT_BUILT, "rt_bvh_get_info: no BVH");
  memset(info, 0, sizeof(*info));
  info->n_prims = s->n_prims;
  info->build_ms = s->last_build_ms;
  info->build_launches = s->last_build_launches;
  if (s->n_prims == 0) return RT_OK;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "rt_bvh_get_info");
  BuildScratch b;
  rt_status rs = carve(s, (int)s->n_prims, b);
  if (rs) return rs;
  if (s->lbvh_cut > 0) {
    // the plain LBVH's cost: refit its nodes above the clusters (once per build;
    // the build's scratch is intact until the next build)
    const int n = (int)s->n_prims;
    k_refit_upper<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n, s->lbvh_cut, b.vals0, b.aabb_lo, b.aabb_hi,
                                                                      b.lch, b.rch, b.parent, b.range, b.node_lo,
                                                                      b.node_hi, b.cost_lbvh, b.flags);
    k_info_sah_lbvh<<<1, 1, 0, (cudaStream_t)stream>>>(b.cost_lbvh, b.info);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_error(e, "rt_bvh_get_info: LBVH cost");
    s->lbvh_cut = 0;
  }
  BuildInfo bi;
  e = cudaMemcpy(&bi, b.info, sizeof(bi), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "rt_bvh_get_info");
  std::vector<float> nodes((size_t)s->n_nodes_total * 16);
  e = cudaMemcpy(nodes.data(), s->nodes.p, nodes.size() * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "rt_bvh_get_info nodes");
  // walk the traversal layout: reachable nodes, depth, leaf sizes, SAH cost
  auto area3 = [](const float* lo, const float* hi) {
    double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1], dz = (double)hi[2] - lo[2];
    if (!(dx >= 0) || !(dy >= 0) || !(dz >= 0)) return 0.0;
    return 2.0 * (dx * dy + dy * dz + dz * dx);
  };
  auto child_box = [&](int node, int c, float* lo, float* hi) {
    const float* n = &nodes[(size_t)node * 16];
    if (c == 0) {
      lo[0] = n[0]; hi[0] = n[1]; lo[1] = n[2]; hi[1] = n[3]; lo[2] = n[8]; hi[2] = n[9];
    } else {
      lo[0] = n[4]; hi[0] = n[5]; lo[1] = n[6]; hi[1] = n[7]; lo[2] = n[10]; hi[2] = n[11];
    }
  };
  auto link_of = [&](int node, int c) {
    int v;
    memcpy(&v, &nodes[(size_t)node * 16 + 12 + c], 4);
    return v;
  };
  float l0[3], h0[3], l1[3], h1[3];
  child_box(s->root, 0, l0, h0);
  child_box(s->root, 1, l1, h1);
  float rlo[3], rhi[3];
  for (int k = 0; k < 3; ++k) {
    rlo[k] = std::min(l0[k], l1[k]);
    rhi[k] = std::max(h0[k], h1[k]);
  }
  double a_root = area3(rlo, rhi);
  double sum = kCostTrav * a_root;
  int64_t reach = 0;
  int max_depth = 0, max_leaf = 0;
  std::vector<std::pair<int, int>> stack;
  stack.push_back({s->root, 1});
  while (!stack.empty()) {
    auto [node, depth] = stack.back();
    stack.pop_back();
    if (node < 0 || node >= s->n_nodes_total || reach > s->n_nodes_total)
      return set_error(RT_ERR_CUDA, "rt_bvh_get_info: malformed tree");
    ++reach;
    max_depth = std::max(max_depth, depth);
    for (int c = 0; c < 2; ++c) {
      float lo[3], hi[3];
      child_box(node, c, lo, hi);
      int link = link_of(node, c);
      if (link < 0) {
        int cnt = leaf_count(link);
        if (s->n_prims == 1 && c == 1) continue;   // the single-primitive root's empty slot
        max_leaf = std::max(max_leaf, cnt);
        sum += kCostIsect * cnt * area3(lo, hi);
      } else {
        sum += kCostTrav * area3(lo, hi);
        stack.push_back({link, depth + 1});
      }
    }
  }
  info->n_nodes = reach;
  info->root = s->root;
  info->max_depth = max_depth;
  info->max_leaf_size = max_leaf;
  info->sah_cost = a_root > 0 ? sum / a_root : 0.0;
  info->sah_cost_lbvh = bi.sah_lbvh;
  return RT_OK;
}

rt_status rt_bvh_export(rt_scene* s, float* nodes, int64_t nodes_capacity, int32_t* prim_order, uint32_t* morton,
                        void* stream) {
  if (!s) return set_error(RT_ERR_INVALID_ARG, "rt_bvh_export: scene is NULL");
  if (!s->built) return set_error(RT_ERR_NOT_BUILT, "rt_bvh_export: no BVH");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "rt_bvh_export");
  int n = (int)s->n_prims;
  if (n == 0) return RT_OK;
  BuildScratch b;
  rt_status rs = carve(s, n, b);
  if (rs) return rs;
  if (nodes) {
    int64_t cnt = std::min<int64_t>(nodes_capacity, s->n_nodes_total);
    e = cudaMemcpy(nodes, s->nodes.p, (size_t)cnt * 64, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "rt_bvh_export nodes");
  }
  if (prim_order) {
    e = cudaMemcpy(prim_order, b.vals0, (size_t)n * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "rt_bvh_export order");
  }
  if (morton) {
    e = cudaMemcpy(morton, b.keys0, (size_t)n * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "rt_bvh_export morton");
    const int drop = 30 - morton_key_bits(n);   // the sort keys are the codes' top bits
    for (int i = 0; i < n; ++i) morton[i] <<= drop;
  }
  return RT_OK;
}

rt_status rt_bvh_export_wide(rt_scene* s, float* nodes, int64_t nodes_capacity, int64_t* n_nodes, void* stream) {
  if (!s) return set_error(RT_ERR_INVALID_ARG, "rt_bvh_export_wide: scene is NULL");
  if (!s->built) return set_error(RT_ERR_NOT_BUILT, "rt_bvh_export_wide: no BVH");
  if (nodes_capacity < 0) return set_error(RT_ERR_INVALID_ARG, "rt_bvh_export_wide: negative capacity");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "rt_bvh_export_wide");
  int64_t slots = s->n_prims > 0 ? s->n_nodes4 : 0;
  if (n_nodes) *n_nodes = slots;
  if (nodes && slots > 0) {
    int64_t cnt = std::min<int64_t>(nodes_capacity, slots);
    e = cudaMemcpy(nodes, s->nodes4.p, (size_t)cnt * 128, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "rt_bvh_export_wide nodes");
  }
  return RT_OK;
}

}  // extern "C"
