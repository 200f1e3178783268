/*
 * oracle.h - FP64 CPU oracle for the Whitted tracer.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does.
 * It shares no code, header or constant with the CUDA sources.
 *
 * What it computes (paper: "Massively Parallel Ray Tracing Algorithm Using
 * GPU", Qin, Lin, Huang):
 *   - ray-sphere hits by the quadratic of Eq. 9-12 (textbook form, in FP64);
 *   - ray-triangle hits (Moller-Trumbore 1997: the plain point-in-plane and
 *     inside-triangle test written with barycentrics);
 *   - local illumination with one shadow ray per point light, Alg. 1 (an
 *     occluder anywhere on the segment blocks the light; otherwise its
 *     irradiance is added once);
 *   - Eq. 8 specialised to point lights and a Lambert + Phong BRDF, plus the
 *     emission term L_e of Eq. 7;
 *   - reflection and refraction rays traced to a fixed depth (Sec. IV.A,
 *     Fig. 3), both recursively and as the paper's iteration-over-depth form.
 *
 * Input arrays use the binary layout of the C ABI structs (4-byte fields,
 * no padding); the oracle promotes every value to double on entry.
 */
#ifndef RTB_ORACLE_H
#define RTB_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_scene orc_scene;

/* Copies and promotes the inputs; builds the oracle's own median-split BVH.
 * background: 3 doubles.  eps_scale: offset scale (1e-4).  fragile_k: the
 * multiplier K of the rounding model (decision margins below K x the
 * modelled FP32 uncertainty are flagged).  Returns NULL on bad input. */
orc_scene* orc_scene_create(const void* spheres, int64_t n_spheres,
                            const void* triangles, int64_t n_triangles,
                            const void* materials, int64_t n_materials,
                            const void* lights, int64_t n_lights,
                            const double* background, double eps_scale,
                            double fragile_k);
void orc_scene_free(orc_scene* s);
int64_t orc_bvh_node_count(const orc_scene* s);

/* Parallelogram area lights (rt_area_light layout: corner, edge_u, edge_v,
 * radiance; 12 floats each), replacing earlier ones; they emit on the side
 * of edge_u x edge_v.  Returns non-zero on a non-finite value or a
 * degenerate parallelogram. */
int orc_set_area_lights(orc_scene* s, const void* lights, int64_t n);

/* The pass that orc_render renders: Philox key `seed`, pass index, strata
 * per axis (S: stratified over S x S passes), and jitter != 0 to move the
 * camera ray to a sampled point of its pixel.  Defaults: seed 0, pass 0,
 * strata 1, no jitter. */
void orc_set_pass(orc_scene* s, uint64_t seed, int32_t pass, int32_t strata, int32_t jitter);

/* Monte-Carlo GI (on != 0): every non-dielectric hit with 1 - rho > 0 and
 * some albedo > 0 spawns, below the last depth, one cosine-weighted diffuse
 * ray of weight pi (1 - rho) albedo (sample slot 2^32 - 2 of its vertex);
 * the ray it makes adds no L_e where it hits.  Default off. */
void orc_set_diffuse_bounce(orc_scene* s, int32_t on);

/* Philox4x32-10 of counter ctr[4] under key key[2] (exposed for tests). */
void orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Pinhole camera ray of pixel (x, y), row 0 at the top.  cam: rt_camera
 * layout (10 floats).  Writes origin o[3] and unit direction d[3]. */
void orc_camera_ray(const void* cam, int width, int height, int x, int y,
                    double* o, double* d);

/* Renders the pixels listed in `pixels` (n_pixels indices y*W+x; NULL =
 * every pixel).  Outputs are indexed like `pixels` (or by pixel when NULL):
 *   rgb[3*i]      radiance (FP64)
 *   prim[i]       primary hit prim id (sphere j -> j, triangle k -> ns+k,
 *                 miss -> -1)
 *   t[i]          primary hit distance (inf on a miss)
 *   robust[i]     smallest decision margin in the pixel's path tree in units
 *                 of the modelled FP32 uncertainty (>= 1: no decision is
 *                 within reach of FP32 rounding)
 *   counts        [3 + 3*(max_depth+1)] ray counts: totals of primary,
 *                 shadow and secondary rays, then per depth (closest-hit
 *                 rays, shadow rays, unused) - may be NULL
 * mode: 0 recursive brute force, 1 recursive with the oracle BVH,
 *       2 iterative (explicit per-depth ray lists, brute force).
 * nthreads <= 0 uses all OpenMP threads.  Returns 0 on success. */
int orc_render(const orc_scene* s, const void* cam, int width, int height,
               int max_depth, int mode, const int64_t* pixels,
               int64_t n_pixels, double* rgb, int32_t* prim, double* t,
               double* robust, uint64_t* counts, int nthreads);

/* orc_render with two more per-pixel outputs (either may be NULL):
 *   robust_struct[i]  smallest margin, in the same units as robust, of any
 *                     decision that changes the pixel's ray counts (which
 *                     primitive a ray hits, front or back, n.l > 0 for a
 *                     light, total internal reflection, the bounce basis),
 *                     taken over every ray whatever its weight; modes 0 and
 *                     1 only
 *   px_counts         n x 2 (max_depth + 1) uint32: per depth d, the
 *                     pixel's closest-hit rays traced at d, then its
 *                     shadow rays cast from depth-d hits */
int orc_render_px(const orc_scene* s, const void* cam, int width, int height,
                  int max_depth, int mode, const int64_t* pixels,
                  int64_t n_pixels, double* rgb, int32_t* prim, double* t,
                  double* robust, uint64_t* counts, double* robust_struct,
                  uint32_t* px_counts, int nthreads);

/* Closest hit for n given FP32 rays (promoted to double), t in (tmin, inf).
 * prim/t as above; robust as above for this single query, with the rays
 * treated as exact (intersection rounding only). */
int orc_closest_hits(const orc_scene* s, int64_t n, const float* o,
                     const float* d, double tmin, int use_bvh, int32_t* prim,
                     double* t, double* robust, int nthreads);

/* Any hit with t in (tmin, tmax[i]) for n given FP32 rays. */
int orc_any_hits(const orc_scene* s, int64_t n, const float* o,
                 const float* d, double tmin, const float* tmax, int use_bvh,
                 uint8_t* occluded, double* robust, int nthreads);

/* Ray-sphere roots of Eq. 11-12 for one sphere; returns the number of real
 * roots (0, 1 or 2), roots ascending in t[0..1]. */
int orc_sphere_roots(const double* o, const double* d, const double* c,
                     double r, double* t);

/* Moller-Trumbore for one triangle: returns 1 on a hit (t > 0) with t, u, v. */
int orc_triangle_hit(const double* o, const double* d, const double* v0,
                     const double* v1, const double* v2, double* t, double* u,
                     double* v);

/* Fresnel-Schlick reflectance and the refracted direction for a unit d
 * meeting a surface with unit normal n facing the ray (d.n < 0).  Returns
 * 1 and writes R and the refracted unit direction, or 0 on total internal
 * reflection (R = 1). */
int orc_refract(const double* d, const double* n, double n1, double n2,
                double* R, double* dt);

/* ---- neural radiance cache oracle (FP64) ---------------------------- */

#define ORC_NRC_NW 18624   /* W0[64][96] W1..W3[64][64] W4[3][64] */
#define ORC_NRC_NB 259     /* b0..b3[64] b4[3] */

/* Renders that follow terminate every hit at depth `depth` (-1: off) with
 * the cache: radiance exp(MLP(encode(p, n, -d))) replaces that hit's local
 * term and children.  Positions are normalised as (p - lo) * inv_ext.
 * bf16 != 0: features and hidden activations rounded to BF16. */
void orc_set_cache(orc_scene* s, int depth, const double* W, const double* B, int bf16, const double* lo,
                   const double* inv_ext);

/* Round to the nearest BF16 value (ties to even), through FP32. */
double orc_round_bf16(double x);

/* Frequency encoding of a hit: 3 normalised position values, normal (3),
 * view direction (3) and sin/cos(2^k pi x_hat) for k = 0..11 (72), i.e.
 * 81 features, zero-padded to 96.  in: n x 9 (p, n, v), bbox: lo[3], hi[3]. */
void orc_nrc_encode(int64_t n, const double* in, const double* bbox_lo,
                    const double* bbox_hi, double* out96);

/* MLP 96 -> 64 -> 64 -> 64 -> 64 -> 3, ReLU hidden, exp output.
 * W: layer weights row-major [out][in] concatenated; B: biases.
 * Layer sizes are fixed by `dims` (6 entries: 96,64,64,64,64,3). */
void orc_mlp_forward(int64_t n, const double* x, const double* W,
                     const double* B, double* y);

/* Mean relative-L2 loss mean((y - t)^2 / (sg(y)^2 + 0.01)) over n x 3 and
 * its gradients dW, dB (same layout as W, B).  Returns the loss. */
double orc_mlp_loss_grad(int64_t n, const double* x, const double* target,
                         const double* W, const double* B, double* dW,
                         double* dB);

/* As above with bf16 != 0: hidden activations rounded to BF16 after the
 * ReLU, and the gradients w.r.t. pre-activations (the backward signal)
 * rounded to BF16 as they are stored, so that the weight, bias and input
 * gradients all use the stored values; the network's activations and
 * backward signals are BF16 by design, the accumulation stays FP64. */
void orc_mlp_forward_ex(int64_t n, const double* x, const double* W, const double* B, double* y, int bf16);
double orc_mlp_loss_grad_ex(int64_t n, const double* x, const double* target, const double* W,
                            const double* B, double* dW, double* dB, int bf16);

/* One Adam step (bias-corrected), in place, on n parameters.  step >= 1. */
void orc_adam(int64_t n, double* w, const double* g, double* m, double* v,
              int64_t step, double lr, double beta1, double beta2, double eps);

#ifdef __cplusplus
}
#endif
#endif
