/*
 * oracle.c - FP64 CPU oracle for the Whitted tracer.
 *
 * TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA path is
 * checked against.  Only the tests, the smoke check and the benchmark's CPU
 * baseline load it.  It shares no code with the CUDA sources.
 *
 * The method (paper: "Massively Parallel Ray Tracing Algorithm Using GPU"):
 *   - Sec. IV.B, Eq. 9-12: a ray o + t d meets a sphere |p - c|^2 = r^2 where
 *     (d.d) t^2 + 2 ((o-c).d) t + (o-c).(o-c) - r^2 = 0, solved with the
 *     quadratic formula.  Triangles (not in the paper) use Moller-Trumbore.
 *   - Alg. 1: at a hit p, one shadow ray per point light; if any object
 *     blocks it the light adds nothing, otherwise its irradiance is added
 *     once (the reading of the garbled per-object IF/ELSE of Alg. 1).
 *   - Eq. 6-8 with point lights: the hemisphere integral of Eq. 8 becomes a
 *     sum over lights; f_r is Lambert (albedo) + Phong (ks, shininess);
 *     L_e of Eq. 7 is the material's emission.
 *   - Sec. IV.A, Fig. 3: each hit spawns, besides the shadow rays, new
 *     reflection / refraction rays; recursion stops at a fixed depth, and the
 *     paper turns the recursion into an iteration over depth.
 * The readings of what the paper leaves open (camera model, offsets,
 * Fresnel-Schlick, background, constants) are stated at each function.
 *
 * Area lights and passes (Sec. IV.A, Alg. 1: the paper samples one point
 * of each light per pass and lets the image converge over passes): a pass
 * k draws, for every path vertex, one stratified point on each
 * parallelogram light and, optionally, a jittered point inside the pixel.
 * The random numbers come from Philox4x32-10 (Salmon et al., "Parallel
 * random numbers: as easy as 1, 2, 3", SC 2011), written here from that
 * definition, keyed by the seed and counted by (pixel, pass, path vertex,
 * slot); the progressive image is the mean of the passes.
 *
 * Monte-Carlo GI (Eq. 8 in full, as an option): besides its light samples a
 * diffuse vertex sends one cosine-weighted ray over its hemisphere, so light
 * that other surfaces reflect reaches it too; the ray it makes adds no L_e
 * where it hits, because the emitters were already sampled as lights.
 *
 * Besides radiance the oracle reports, per pixel, how close any decision in
 * the pixel's path tree (which primitive is hit, whether a light is blocked,
 * front/back side, n.l > 0, total internal reflection) comes to flipping,
 * measured in units of a first-order model of FP32 rounding.  That number
 * is diagnostic only; it never changes the radiance.
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GAMMA32 5.9604644775390625e-08 /* 2^-24, FP32 unit roundoff */
#define ROBUST_CAP 1.0e6
#define LEAF_MAX 4
#define STACK_MAX 256
#define MAX_DEPTH_LIMIT 16

/* ------------------------------------------------------------------ */
/* small vector algebra                                                */
/* ------------------------------------------------------------------ */
typedef struct { double x, y, z; } v3;
static inline v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static inline v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static inline v3 mul(v3 a, v3 b) { return mk(a.x * b.x, a.y * b.y, a.z * b.z); }
static inline double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline v3 cross(v3 a, v3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static inline double len(v3 a) { return sqrt(dot(a, a)); }
static inline v3 unit(v3 a) { return scl(a, 1.0 / len(a)); }
static inline double maxabs(v3 a) {
  double m = fabs(a.x);
  if (fabs(a.y) > m) m = fabs(a.y);
  if (fabs(a.z) > m) m = fabs(a.z);
  return m;
}
static inline double maxc(v3 a) { return fmax(a.x, fmax(a.y, a.z)); }
static inline v3 vmin(v3 a, v3 b) { return mk(fmin(a.x, b.x), fmin(a.y, b.y), fmin(a.z, b.z)); }
static inline v3 vmax(v3 a, v3 b) { return mk(fmax(a.x, b.x), fmax(a.y, b.y), fmax(a.z, b.z)); }
static inline double comp(v3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }
static inline v3 f3(const float* p) { return mk(p[0], p[1], p[2]); }

/* ------------------------------------------------------------------ */
/* input layouts (same bytes as the C ABI structs)                      */
/* ------------------------------------------------------------------ */
typedef struct { float c[3]; float r; uint32_t mat; } in_sphere;
typedef struct { float v0[3], v1[3], v2[3]; uint32_t mat; } in_tri;
typedef struct {
  uint32_t kind; float albedo[3]; float ks, shininess, reflectivity, ior; float emission[3];
} in_mat;
typedef struct { float pos[3]; float intensity[3]; } in_light;
typedef struct { float eye[3], look_at[3], up[3]; float vfov_deg; } in_cam;

enum { KIND_DIFFUSE = 0, KIND_MIRROR = 1, KIND_DIELECTRIC = 2 };

typedef struct {
  int is_sphere;
  uint32_t mat;
  v3 c; double r;      /* sphere */
  v3 v0, v1, v2;       /* triangle */
  v3 lo, hi, centroid;
  double scale;        /* largest |coordinate| of the primitive */
  double aspect;       /* longest edge / smallest altitude (conditioning of the normal) */
  v3 bc; double brad;  /* bounding sphere (centre, radius) */
} prim_t;

typedef struct { uint32_t kind; v3 albedo; double ks, shin, refl, ior; v3 emis; } mat_t;
typedef struct { v3 pos, inten; } light_t;
/* parallelogram light corner + a eu + b ev (a, b in [0, 1]); emits L on the
 * side of nl = unit(eu x ev) */
typedef struct { v3 corner, eu, ev, L, nl; double area; } alight_t;
typedef struct { float corner[3], edge_u[3], edge_v[3], radiance[3]; } in_alight;
typedef struct { v3 lo, hi; int64_t left, right, start, count; } node_t;

struct orc_scene {
  int64_t n_prims, n_spheres;
  prim_t* prims;
  int64_t n_mats; mat_t* mats;
  int64_t n_lights; light_t* lights;
  int64_t n_alights; alight_t* alights;
  int64_t n_emitters; int64_t* emitters;   /* primitives whose material emits (Eq. 7), sampled as lights */
  /* the pass being rendered: Philox key, pass index, strata per axis, and
   * whether the camera ray is jittered inside its pixel */
  uint32_t seed_lo, seed_hi;
  int32_t pass, strata, jitter;
  int32_t bounce;      /* Monte-Carlo GI: one cosine-weighted diffuse bounce per vertex */
  v3 bg;
  double eps_scale, K;
  double l_max;        /* bound on the radiance any subtree returns */
  v3 scene_lo, scene_hi;
  int64_t n_nodes; node_t* nodes; int64_t* order;
  /* radiance cache (nrc_depth < 0: none): network parameters and box */
  int nrc_depth, nrc_bf16;
  double* nrc_W;
  double* nrc_B;
  double nrc_lo[3], nrc_inv_ext[3];
};

/* A ray with the modelled FP32 uncertainty of its origin (absolute, eo),
 * of its origin across the surface it left (en; what decides whether the
 * ray re-hits that surface) and of its direction (radians, ed); see the
 * rounding model below. */
typedef struct { v3 o, d; double eo, ed, en; } ray_t;

/* ------------------------------------------------------------------ */
/* rounding model (diagnostic)                                          */
/*                                                                      */
/* U(t) is the positional uncertainty, at distance t along the ray, of   */
/* an FP32 implementation of the same arithmetic: K * 2^-24 * (|o| + t + */
/* |prim|) plus the uncertainty the ray inherited.  A decision whose     */
/* margin (a distance, or an angle for the shading tests) is below the   */
/* uncertainty it is compared against has robust < 1.                   */
/* ------------------------------------------------------------------ */
static inline double unc(const orc_scene* s, const ray_t* r, double t, double prim_scale) {
  double tt = t > 0 && isfinite(t) ? t : 0.0;
  return s->K * GAMMA32 * (maxabs(r->o) + tt + prim_scale) + r->eo + r->ed * tt;
}

/* uncertainty of decisions taken right at the origin (t near tmin) */
static inline double unc0(const orc_scene* s, const ray_t* r, double prim_scale) {
  return s->K * GAMMA32 * (maxabs(r->o) + prim_scale) + r->en;
}

/* Per-primitive test result for one ray. */
typedef struct {
  int hit;        /* the exact test passes with t > tmin */
  int inside;     /* barycentric / discriminant test passes (any t) */
  double t;       /* hit distance; for a miss, where the ray passes closest */
  double t_lo;    /* sphere: smaller root (or t) */
  double margin;  /* distance to the hit/miss boundary, conditioned (>= 0) */
  double cosn;    /* |cos| between the ray and the surface normal there */
} cand_t;

/* Ray-sphere, Eq. 11-12: a = d.d, b = 2 (o-c).d, c = (o-c).(o-c) - r^2,
 * t = (-b +- sqrt(b^2 - 4ac)) / 2a.  The nearer root above tmin is the hit;
 * from inside the sphere that is the larger root. */
static cand_t sphere_cand(const prim_t* p, v3 o, v3 d, double tmin) {
  cand_t c;
  memset(&c, 0, sizeof c);
  v3 f = sub(o, p->c);
  double a = dot(d, d);
  double b = 2.0 * dot(f, d);
  double cc = dot(f, f) - p->r * p->r;
  double disc = b * b - 4.0 * a * cc;
  double tca = -dot(f, d) / a;                 /* closest approach */
  double dist = len(sub(f, scl(d, dot(f, d) / a)));
  if (disc < 0.0) {
    c.t = tca; c.t_lo = tca;
    c.margin = dist - p->r;
    if (c.margin < 0) c.margin = 0;
    return c;
  }
  c.inside = 1;
  double sq = sqrt(disc);
  double t0 = (-b - sq) / (2.0 * a);
  double t1 = (-b + sq) / (2.0 * a);
  c.t_lo = t0;
  c.margin = p->r - dist;
  if (c.margin < 0) c.margin = 0;
  if (t0 > tmin) { c.hit = 1; c.t = t0; }
  else if (t1 > tmin) { c.hit = 1; c.t = t1; }
  else c.t = t1;
  v3 ph = add(o, scl(d, c.t));
  c.cosn = fabs(dot(d, sub(ph, p->c))) / (p->r * sqrt(a));
  return c;
}

/* Moller-Trumbore (1997): edges e1 = v1-v0, e2 = v2-v0; P = d x e2,
 * det = e1.P; T = o - v0; u = T.P/det; Q = T x e1; v = d.Q/det;
 * t = e2.Q/det.  Hit iff det != 0, u >= 0, v >= 0, u + v <= 1, t > tmin
 * (two-sided; edges inclusive). */
static cand_t tri_cand(const prim_t* p, v3 o, v3 d, double tmin) {
  cand_t c;
  memset(&c, 0, sizeof c);
  v3 e1 = sub(p->v1, p->v0), e2 = sub(p->v2, p->v0);
  v3 P = cross(d, e2);
  double det = dot(e1, P);
  if (det == 0.0) { c.t = INFINITY; c.t_lo = INFINITY; c.margin = INFINITY; return c; }
  double inv = 1.0 / det;
  v3 T = sub(o, p->v0);
  double u = dot(T, P) * inv;
  v3 Q = cross(T, e1);
  double v = dot(d, Q) * inv;
  double t = dot(e2, Q) * inv;
  double w = 1.0 - u - v;
  c.t = t; c.t_lo = t;
  c.inside = (u >= 0.0 && v >= 0.0 && u + v <= 1.0);
  c.hit = c.inside && t > tmin;
  /* Distance of the ray line to each edge line times the sine of the angle
   * between them: bary * |det| / |edge| (for unit d). */
  double adet = fabs(det) / len(d);
  double du = u * adet / len(e2);
  double dv = v * adet / len(e1);
  double dw = w * adet / len(sub(e2, e1));
  if (c.inside) {
    c.margin = fmin(du, fmin(dv, dw));
  } else {
    double m = 0;
    if (-du > m) m = -du;
    if (-dv > m) m = -dv;
    if (-dw > m) m = -dw;
    c.margin = m;
  }
  c.cosn = fabs(det) / (len(cross(e1, e2)) * len(d));
  return c;
}

static inline cand_t prim_cand(const prim_t* p, v3 o, v3 d, double tmin) {
  return p->is_sphere ? sphere_cand(p, o, d, tmin) : tri_cand(p, o, d, tmin);
}

/* ------------------------------------------------------------------ */
/* the oracle's own BVH: median split over centroids, <= 4 prims a leaf */
/* ------------------------------------------------------------------ */
static int g_sort_axis;
static const prim_t* g_sort_prims;
static int cmp_centroid(const void* a, const void* b) {
  int64_t i = *(const int64_t*)a, j = *(const int64_t*)b;
  double ci = comp(g_sort_prims[i].centroid, g_sort_axis);
  double cj = comp(g_sort_prims[j].centroid, g_sort_axis);
  if (ci < cj) return -1;
  if (ci > cj) return 1;
  return (i > j) - (i < j);
}

static int64_t bvh_build_rec(orc_scene* s, int64_t start, int64_t count) {
  int64_t me = s->n_nodes++;
  node_t* n = &s->nodes[me];
  v3 lo = mk(INFINITY, INFINITY, INFINITY), hi = mk(-INFINITY, -INFINITY, -INFINITY);
  v3 clo = lo, chi = hi;
  for (int64_t i = start; i < start + count; ++i) {
    const prim_t* p = &s->prims[s->order[i]];
    lo = vmin(lo, p->lo); hi = vmax(hi, p->hi);
    clo = vmin(clo, p->centroid); chi = vmax(chi, p->centroid);
  }
  n->lo = lo; n->hi = hi;
  if (count <= LEAF_MAX) {
    n->start = start; n->count = count; n->left = n->right = -1;
    return me;
  }
  v3 ext = sub(chi, clo);
  int axis = (ext.x >= ext.y && ext.x >= ext.z) ? 0 : (ext.y >= ext.z ? 1 : 2);
  g_sort_axis = axis;
  g_sort_prims = s->prims;
  qsort(s->order + start, (size_t)count, sizeof(int64_t), cmp_centroid);
  int64_t half = count / 2;
  n->count = 0; n->start = -1;
  int64_t l = bvh_build_rec(s, start, half);
  int64_t r = bvh_build_rec(s, start + half, count - half);
  s->nodes[me].left = l;
  s->nodes[me].right = r;
  return me;
}

/* slab test of the ray segment [t0, t1] against a box grown by m */
static int box_overlap(v3 lo, v3 hi, double m, const ray_t* r, double t0, double t1) {
  for (int k = 0; k < 3; ++k) {
    double o = comp(r->o, k), d = comp(r->d, k);
    double a = comp(lo, k) - m, b = comp(hi, k) + m;
    if (d == 0.0) {
      if (o < a || o > b) return 0;
      continue;
    }
    double ta = (a - o) / d, tb = (b - o) / d;
    if (ta > tb) { double x = ta; ta = tb; tb = x; }
    if (ta > t0) t0 = ta;
    if (tb < t1) t1 = tb;
    if (t0 > t1) return 0;
  }
  return 1;
}

/* Visits every primitive whose (grown) box meets the segment; calls fn. */
typedef void (*visit_fn)(void* ctx, int64_t prim);
static void bvh_visit(const orc_scene* s, const ray_t* r, double t0, double t1, double m,
                      visit_fn fn, void* ctx) {
  int64_t stack[STACK_MAX];
  int sp = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const node_t* n = &s->nodes[stack[--sp]];
    if (!box_overlap(n->lo, n->hi, m, r, t0, t1)) continue;
    if (n->count > 0) {
      for (int64_t i = n->start; i < n->start + n->count; ++i) fn(ctx, s->order[i]);
    } else {
      stack[sp++] = n->left;
      stack[sp++] = n->right;
    }
  }
}

/* ------------------------------------------------------------------ */
/* closest hit and any hit, with decision margins                       */
/* ------------------------------------------------------------------ */
typedef struct {
  const orc_scene* s;
  const ray_t* r;
  double tmin;
  int32_t best;
  double best_t, best_cos;
  double robust;
} ch_ctx;

static void ch_best_visit(void* vc, int64_t i) {
  ch_ctx* c = (ch_ctx*)vc;
  cand_t h = prim_cand(&c->s->prims[i], c->r->o, c->r->d, c->tmin);
  if (!h.hit) return;
  /* nearest t; equal t goes to the lower primitive id */
  if (h.t < c->best_t || (h.t == c->best_t && (int32_t)i < c->best)) {
    c->best = (int32_t)i; c->best_t = h.t; c->best_cos = h.cosn;
  }
}

/* Where along the ray a missed primitive is passed: its plane / closest
 * approach t, clamped to the span of its bounding sphere. */
static double t_near(const prim_t* p, const ray_t* r, double t) {
  double tc = dot(sub(p->bc, r->o), r->d) / dot(r->d, r->d);
  double rr = p->brad / len(r->d);
  if (t < tc - rr) t = tc - rr;
  if (t > tc + rr) t = tc + rr;
  return t;
}

static void ch_robust_visit(void* vc, int64_t i) {
  ch_ctx* c = (ch_ctx*)vc;
  const prim_t* p = &c->s->prims[i];
  cand_t h = prim_cand(p, c->r->o, c->r->d, c->tmin);
  double rb = ROBUST_CAP;
  if ((int32_t)i == c->best) {
    double u = unc(c->s, c->r, h.t, p->scale);
    rb = h.margin / u;                                   /* the hit could be lost */
    double u0 = unc0(c->s, c->r, p->scale);
    double near0 = (h.t - c->tmin) * h.cosn / u0;        /* hit right at the origin */
    if (near0 < rb) rb = near0;
    if (p->is_sphere && h.t_lo <= c->tmin && h.t != h.t_lo) {
      double r2 = (c->tmin - h.t_lo) * h.cosn / u0;      /* other root near the origin */
      if (r2 < rb) rb = r2;
    }
  } else if (h.hit) {
    /* a farther (or equal-t, higher-id) hit: near-tie in t */
    double u = unc(c->s, c->r, c->best_t, p->scale);
    double cs = fmax(fmin(h.cosn, c->best_cos), 1e-3);
    rb = (h.t - c->best_t) / (1e-6 * c->best_t + u / cs);
  } else if (h.inside) {
    /* inside the test but at t <= tmin: behind or at the origin */
    double u0 = unc0(c->s, c->r, p->scale);
    rb = (c->tmin - h.t) * fmax(h.cosn, 1e-3) / u0;
    if (rb < 0) rb = 0;
  } else if (isfinite(h.t)) {
    /* missed, but passing near it in front of the nearest hit */
    double te = t_near(p, c->r, h.t);
    if (te > c->tmin && te <= c->best_t) rb = h.margin / unc(c->s, c->r, te, p->scale);
  }
  if (rb < c->robust) c->robust = rb;
}

typedef struct { int32_t prim; double t, cosn, robust; } hit_t;

static double ray_extent(const orc_scene* s, const ray_t* r) {
  /* farthest t at which the ray can still be inside the scene box */
  double te = 0;
  for (int k = 0; k < 8; ++k) {
    v3 c = mk(k & 1 ? s->scene_hi.x : s->scene_lo.x, k & 2 ? s->scene_hi.y : s->scene_lo.y,
              k & 4 ? s->scene_hi.z : s->scene_lo.z);
    double d = len(sub(c, r->o));
    if (d > te) te = d;
  }
  return te / len(r->d) + 1.0;
}

static hit_t closest_hit(const orc_scene* s, const ray_t* r, double tmin, int use_bvh, int want_robust) {
  ch_ctx c;
  c.s = s; c.r = r; c.tmin = tmin; c.best = -1; c.best_t = INFINITY; c.best_cos = 1.0;
  c.robust = ROBUST_CAP;
  if (use_bvh && s->n_nodes > 0) {
    double m1 = 1e-12 * (maxabs(s->scene_lo) + maxabs(s->scene_hi) + 1.0);
    bvh_visit(s, r, -INFINITY, INFINITY, m1, ch_best_visit, &c);
  } else {
    for (int64_t i = 0; i < s->n_prims; ++i) ch_best_visit(&c, i);
  }
  if (want_robust) {
    if (use_bvh && s->n_nodes > 0) {
      double tl = c.best >= 0 ? c.best_t : ray_extent(s, r);
      double m = 640.0 * unc(s, r, tl, maxabs(s->scene_lo) + maxabs(s->scene_hi));
      bvh_visit(s, r, tmin - m, tl + m, m, ch_robust_visit, &c);
    } else {
      for (int64_t i = 0; i < s->n_prims; ++i) ch_robust_visit(&c, i);
    }
  }
  hit_t h = {c.best, c.best_t, c.best_cos, c.robust};
  return h;
}

typedef struct {
  const orc_scene* s;
  const ray_t* r;
  double tmin, tmax;
  int occluded;
  double best_occ;     /* strongest occluder's margin */
  double near_miss;    /* smallest margin of a non-occluder */
} ah_ctx;

static void ah_visit(void* vc, int64_t i) {
  ah_ctx* c = (ah_ctx*)vc;
  const prim_t* p = &c->s->prims[i];
  cand_t h = prim_cand(p, c->r->o, c->r->d, c->tmin);
  /* A sphere may have its second root inside the segment */
  double t = h.t;
  int occ = h.hit && t < c->tmax;
  if (occ) {
    c->occluded = 1;
    double u = unc(c->s, c->r, t, p->scale);
    double cs = fmax(h.cosn, 1e-3);
    double m = h.margin / u;
    double m2 = (c->tmax - t) * cs / u;
    double m3 = (t - c->tmin) * cs / unc0(c->s, c->r, p->scale);
    if (m2 < m) m = m2;
    if (m3 < m) m = m3;
    if (m > c->best_occ) c->best_occ = m;
  } else {
    double rb = ROBUST_CAP;
    if (h.inside && isfinite(t)) {
      double u = unc(c->s, c->r, t, p->scale);
      double cs = fmax(h.cosn, 1e-3);
      if (h.hit) rb = (t - c->tmax) * cs / u;                /* just beyond the light */
      else rb = (c->tmin - t) * cs / unc0(c->s, c->r, p->scale); /* just behind the origin */
      if (rb < 0) rb = 0;
    } else if (!h.inside && isfinite(t)) {
      double te = t_near(p, c->r, t);
      if (te > c->tmin && te < c->tmax) rb = h.margin / unc(c->s, c->r, te, p->scale);
    }
    if (rb < c->near_miss) c->near_miss = rb;
  }
}

static int any_hit(const orc_scene* s, const ray_t* r, double tmin, double tmax, int use_bvh,
                   double* robust) {
  ah_ctx c;
  c.s = s; c.r = r; c.tmin = tmin; c.tmax = tmax; c.occluded = 0;
  c.best_occ = 0.0; c.near_miss = ROBUST_CAP;
  if (use_bvh && s->n_nodes > 0) {
    double m = 640.0 * unc(s, r, tmax, maxabs(s->scene_lo) + maxabs(s->scene_hi));
    bvh_visit(s, r, tmin - m, tmax + m, m, ah_visit, &c);
  } else {
    for (int64_t i = 0; i < s->n_prims; ++i) ah_visit(&c, i);
  }
  if (robust) *robust = c.occluded ? c.best_occ : c.near_miss;
  return c.occluded;
}

/* ------------------------------------------------------------------ */
/* surface geometry and optics                                          */
/* ------------------------------------------------------------------ */
static v3 geometric_normal(const prim_t* p, v3 ph) {
  if (p->is_sphere) return scl(sub(ph, p->c), 1.0 / p->r);
  return unit(cross(sub(p->v1, p->v0), sub(p->v2, p->v0)));
}

/* Offset of secondary and shadow origins: eps = eps_scale * max(1, |p|_inf)
 * (the paper gives none). */
static inline double offset_eps(const orc_scene* s, v3 p) { return s->eps_scale * fmax(1.0, maxabs(p)); }

static inline v3 reflect(v3 d, v3 n) { return sub(d, scl(n, 2.0 * dot(d, n))); }

/* Snell refraction of unit d through unit n (d.n < 0), eta = n1/n2, and the
 * Fresnel-Schlick reflectance R = R0 + (1-R0)(1-cos)^5 with
 * R0 = ((n1-n2)/(n1+n2))^2 and cos the cosine on the less dense side.
 * Returns 0 on total internal reflection. */
static int refract_schlick(v3 d, v3 n, double n1, double n2, double* R, v3* dt, double* kk) {
  double eta = n1 / n2;
  double ci = -dot(d, n);
  double k = 1.0 - eta * eta * (1.0 - ci * ci);
  if (kk) *kk = k;
  if (k < 0.0) { *R = 1.0; return 0; }
  double ct = sqrt(k);
  *dt = unit(add(scl(d, eta), scl(n, eta * ci - ct)));
  double r0 = (n1 - n2) / (n1 + n2);
  r0 *= r0;
  double c = (n1 <= n2) ? ci : ct;
  double x = 1.0 - c;
  *R = r0 + (1.0 - r0) * x * x * x * x * x;
  return 1;
}

/* ------------------------------------------------------------------ */
/* shading: one hit                                                     */
/* ------------------------------------------------------------------ */
/* ------------------------------------------------------------------ */
/* Philox4x32-10: ten rounds of two 32x32 -> 64-bit products whose high   */
/* halves are mixed with the other counter words and the round key; the  */
/* key grows by the Weyl constants after every round.                    */
/* ------------------------------------------------------------------ */
void orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in [0, 1) from the top 24 bits (exact in FP32 and FP64) */
static inline double unit24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

#define SLOT_PIXEL 0xFFFFFFFFu
#define SLOT_BOUNCE 0xFFFFFFFEu
/* bit 31 of a path-vertex code marks a ray made by a diffuse bounce; the
 * other bits number the vertex (1 for the camera ray, 2c and 2c + 1 for
 * the children of vertex c) */
#define CODE_BOUNCE 0x80000000u

/* A stratified 2-D sample of pass k for (pixel, path vertex `code`, slot):
 * over S x S consecutive passes each cell of an S x S grid is visited once,
 * starting from a cell chosen per pixel and vertex; the point is uniform in
 * its cell. */
static void pass_sample(const orc_scene* s, int64_t pixel, uint32_t code, uint32_t slot, double* a, double* b) {
  uint32_t key[2] = {s->seed_lo, s->seed_hi}, r[4], q[4];
  uint32_t ctr[4] = {(uint32_t)pixel, (uint32_t)s->pass, code, slot};
  orc_philox4x32(ctr, key, r);
  /* the first cell of this (pixel, vertex, slot): the same in every pass */
  uint32_t ctr0[4] = {(uint32_t)pixel, 0xFFFFFFFFu, code, slot};
  orc_philox4x32(ctr0, key, q);
  uint32_t S = (uint32_t)(s->strata > 0 ? s->strata : 1), cells = S * S;
  uint32_t cell = ((uint32_t)s->pass % cells + q[0] % cells) % cells;
  *a = ((double)(cell % S) + unit24(r[0])) / (double)S;
  *b = ((double)(cell / S) + unit24(r[1])) / (double)S;
}

typedef struct { v3 o, d; v3 w; ray_t r; uint32_t code; } child_t;

/* A cosine-weighted direction about the unit normal n for (a, b) in
 * [0, 1)^2 (Malley's method: the point (sqrt(a), 2 pi b) of the unit disk in
 * polar form, lifted onto the hemisphere), expressed in the branch-free
 * orthonormal basis of Duff et al., "Building an Orthonormal Basis,
 * Revisited" (JCGT 2017), with the sign taken as n.z >= 0. */
static v3 cosine_dir(v3 n, double a, double b) {
  double sg = n.z >= 0.0 ? 1.0 : -1.0;
  double k = -1.0 / (sg + n.z);
  double m = n.x * n.y * k;
  v3 t1 = mk(1.0 + sg * n.x * n.x * k, sg * m, -sg * n.x);
  v3 t2 = mk(m, sg + n.y * n.y * k, -n.y);
  double r = sqrt(a), phi = 2.0 * M_PI * b;
  return unit(add(add(scl(t1, r * cos(phi)), scl(t2, r * sin(phi))), scl(n, sqrt(fmax(0.0, 1.0 - a)))));
}

typedef struct {
  v3 local;            /* emission + (1 - rho) * sum over unblocked lights */
  int n_children;
  child_t child[2];
  double robust;
  double robust_struct; /* smallest margin of a decision that changes the ray counts, any weight */
  int n_shadow;
} shade_t;

/* Shades a hit of ray r (weight w) on primitive `pi` at distance t.  The
 * returned local term is already weighted by w; children carry their own
 * absolute weights.  spawn = 0 at the last depth. */
static shade_t shade_hit(const orc_scene* s, const ray_t* r, v3 w, int32_t pi, double t, double hit_cos,
                         int spawn, int use_bvh, int want_robust, int64_t pixel, uint32_t code) {
  shade_t out;
  memset(&out, 0, sizeof out);
  out.robust = ROBUST_CAP;
  out.robust_struct = ROBUST_CAP;
  const prim_t* p = &s->prims[pi];
  const mat_t* m = &s->mats[p->mat];
  v3 ph = add(r->o, scl(r->d, t));
  v3 ng = geometric_normal(p, ph);
  double wmax = maxc(w);
  int count_robust = want_robust && wmax * s->l_max >= 1e-3;

  /* modelled uncertainties at the hit */
  double U = unc(s, r, t, p->scale);
  double Up = U / fmax(hit_cos, 1e-3);                   /* hit point along the surface */
  double An = p->is_sphere ? Up / p->r + s->K * 4 * GAMMA32
                           : s->K * 4 * GAMMA32 * (p->aspect + 1.0);
  double Ad = r->ed + An + s->K * 4 * GAMMA32;

  /* front / back (Sec. IV.A needs inside/outside for refraction) */
  double dn = dot(r->d, ng);
  int inside = dn > 0.0;
  v3 n = inside ? scl(ng, -1.0) : ng;
  if (want_robust) {
    double rb = fabs(dn) / Ad;
    if (count_robust && rb < out.robust) out.robust = rb;
    if (rb < out.robust_struct) out.robust_struct = rb;
  }

  /* L_e of Eq. 7, except on a ray made by a diffuse bounce: the vertex
   * that bounced sampled every emitter as a light already */
  const int via_bounce = (code & CODE_BOUNCE) != 0;
  code &= ~CODE_BOUNCE;
  out.local = via_bounce ? mk(0.0, 0.0, 0.0) : mul(w, m->emis);

  double eps = offset_eps(s, ph);
  v3 o_up = add(ph, scl(n, eps));
  double eo_child = Up + s->K * GAMMA32 * maxabs(ph);
  /* Whatever the ray's own uncertainty, the computed hit lies on the
   * surface up to the rounding of the hit arithmetic alone. */
  double en_child = s->K * GAMMA32 * (maxabs(r->o) + t + p->scale + maxabs(ph));

  if (m->kind != KIND_DIELECTRIC) {
    double rho = m->kind == KIND_MIRROR ? m->refl : 0.0;
    if (1.0 - rho > 0.0) {
      /* Alg. 1: one shadow ray per point light (Eq. 8 with point lights) */
      for (int64_t li = 0; li < s->n_lights; ++li) {
        const light_t* L = &s->lights[li];
        v3 l = unit(sub(L->pos, ph));
        double nl = dot(n, l);
        double dist_l = len(sub(L->pos, ph));
        v3 vdir = scl(r->d, -1.0);
        v3 rl = sub(scl(n, 2.0 * nl), l);                  /* reflect(-l, n) */
        double rv = dot(rl, vdir);
        double spec = rv > 0.0 ? pow(rv, m->shin) : 0.0;
        v3 f = add(scl(m->albedo, nl), mk(m->ks * spec, m->ks * spec, m->ks * spec));
        v3 contrib = scl(mul(mul(w, L->inten), f), 1.0 - rho);
        int relevant = count_robust && maxc(mul(scl(w, 1.0 - rho), L->inten)) * (2.0 + m->ks) >= 1e-3;
        if (want_robust) {
          /* n.l > 0 decides whether a shadow ray is cast */
          double rb = fabs(nl) / (An + r->ed + (Up + s->K * GAMMA32 * maxabs(L->pos)) / dist_l);
          if (relevant && rb < out.robust) out.robust = rb;
          if (rb < out.robust_struct) out.robust_struct = rb;
        }
        if (!(nl > 0.0)) continue;
        /* shadow ray from the offset origin to the light */
        ray_t sr;
        sr.o = o_up;
        v3 to_l = sub(L->pos, o_up);
        double dist = len(to_l);
        sr.d = scl(to_l, 1.0 / dist);
        sr.eo = eo_child;
        sr.en = en_child;
        sr.ed = (eo_child + s->K * GAMMA32 * maxabs(L->pos)) / dist + s->K * 4 * GAMMA32;
        out.n_shadow++;
        double rb = ROBUST_CAP;
        int occ = any_hit(s, &sr, 0.0, dist - eps, use_bvh, relevant && maxc(contrib) >= 1e-3 ? &rb : NULL);
        if (relevant && maxc(contrib) >= 1e-3 && rb < out.robust) out.robust = rb;
        if (!occ) out.local = add(out.local, contrib);
      }
      /* area lights, then emissive primitives (Eq. 7's L_e as a light): one
       * stratified point on each per pass, the same term as a point light
       * times A cos(theta_y) / r^2 (Eq. 8 over the light's area, sampled
       * with density 1 / A) */
      for (int64_t li = 0; li < s->n_alights + s->n_emitters; ++li) {
        double a, b;
        pass_sample(s, pixel, code, (uint32_t)li, &a, &b);
        v3 y, ny, Lrad;
        double area;
        int two_sided = 0;
        if (li < s->n_alights) {
          const alight_t* A = &s->alights[li];
          y = add(A->corner, add(scl(A->eu, a), scl(A->ev, b)));
          ny = A->nl;
          Lrad = A->L;
          area = A->area;
        } else {
          const prim_t* E = &s->prims[s->emitters[li - s->n_alights]];
          Lrad = s->mats[E->mat].emis;
          if (E->is_sphere) {
            /* uniform on the sphere: z = 1 - 2a, azimuth 2 pi b */
            double z = 1.0 - 2.0 * a, rho_xy = sqrt(fmax(0.0, 1.0 - z * z)), phi = 2.0 * M_PI * b;
            ny = mk(rho_xy * cos(phi), rho_xy * sin(phi), z);
            y = add(E->c, scl(ny, E->r));
            area = 4.0 * M_PI * E->r * E->r;
          } else {
            /* uniform on the triangle: fold (a, b) into a + b <= 1 */
            if (a + b > 1.0) { a = 1.0 - a; b = 1.0 - b; }
            v3 e1 = sub(E->v1, E->v0), e2 = sub(E->v2, E->v0), c = cross(e1, e2);
            y = add(E->v0, add(scl(e1, a), scl(e2, b)));
            area = 0.5 * len(c);
            ny = unit(c);
            two_sided = 1;   /* triangles emit (and are hit) on both sides */
          }
        }
        v3 to = sub(y, ph);
        double dist_c = len(to);
        v3 l = scl(to, 1.0 / dist_c);
        double nl = dot(n, l);
        double cos_y = -dot(l, ny);
        if (two_sided) cos_y = fabs(cos_y);
        v3 vdir = scl(r->d, -1.0);
        v3 rl = sub(scl(n, 2.0 * nl), l);                  /* reflect(-l, n) */
        double rv = dot(rl, vdir);
        double spec = rv > 0.0 ? pow(rv, m->shin) : 0.0;
        v3 f = add(scl(m->albedo, nl), mk(m->ks * spec, m->ks * spec, m->ks * spec));
        double G = area * cos_y / (dist_c * dist_c);
        v3 contrib = scl(mul(mul(w, Lrad), f), G * (1.0 - rho));
        double uy = (Up + s->K * 3 * GAMMA32 * maxabs(y)) / dist_c;   /* direction to the sample */
        int relevant = count_robust && maxc(scl(mul(w, Lrad), (1.0 - rho) * fabs(G))) * (2.0 + m->ks) >= 1e-3;
        if (want_robust) {
          double rb = fabs(nl) / (An + r->ed + uy);
          double rb2 = fabs(cos_y) / (uy + s->K * 8 * GAMMA32);
          if (rb2 < rb) rb = rb2;
          if (relevant && rb < out.robust) out.robust = rb;
          if (rb < out.robust_struct) out.robust_struct = rb;
        }
        if (!(nl > 0.0) || !(cos_y > 0.0)) continue;
        ray_t sr;
        sr.o = o_up;
        v3 to_y = sub(y, o_up);
        double dist = len(to_y);
        sr.d = scl(to_y, 1.0 / dist);
        sr.eo = eo_child;
        sr.en = en_child;
        sr.ed = (eo_child + s->K * 3 * GAMMA32 * maxabs(y)) / dist + s->K * 4 * GAMMA32;
        out.n_shadow++;
        double rb = ROBUST_CAP;
        int occ = any_hit(s, &sr, 0.0, dist - eps, use_bvh, relevant && maxc(contrib) >= 1e-3 ? &rb : NULL);
        if (relevant && maxc(contrib) >= 1e-3 && rb < out.robust) out.robust = rb;
        if (!occ) out.local = add(out.local, contrib);
      }
    }
    if (spawn && rho > 0.0) {
      child_t* c = &out.child[out.n_children++];
      c->r.o = o_up;
      c->r.d = unit(reflect(r->d, n));
      c->r.eo = eo_child;
      c->r.en = en_child;
      c->r.ed = r->ed + 2.0 * An + s->K * 8 * GAMMA32;
      c->w = scl(w, rho);
      c->code = code << 1;
    }
    /* Monte-Carlo GI (Eq. 8's hemisphere integral): one cosine-weighted
     * diffuse bounce; with f_r = albedo (the albedo convention of the light
     * terms) and density cos / pi its weight is pi (1 - rho) albedo.  Only
     * the Lambert lobe is integrated: the Phong lobe stays a light term. */
    if (spawn && s->bounce && 1.0 - rho > 0.0 && maxc(m->albedo) > 0.0) {
      double a, b;
      pass_sample(s, pixel, code, SLOT_BOUNCE, &a, &b);
      child_t* c = &out.child[out.n_children++];
      c->r.o = o_up;
      c->r.d = cosine_dir(n, a, b);
      c->r.eo = eo_child;
      c->r.en = en_child;
      c->r.ed = 3.0 * An + s->K * 16 * GAMMA32;
      c->w = scl(mul(w, m->albedo), M_PI * (1.0 - rho));
      c->code = ((code << 1) | 1u) | CODE_BOUNCE;
      if (want_robust) {
        /* the basis changes branch where n.z changes sign */
        double rb = fabs(n.z) / (An + s->K * 4 * GAMMA32);
        if (count_robust && rb < out.robust) out.robust = rb;
        if (rb < out.robust_struct) out.robust_struct = rb;
      }
    }
  } else {
    double n1 = inside ? m->ior : 1.0, n2 = inside ? 1.0 : m->ior;
    double R, kk;
    v3 dt;
    int has_t = refract_schlick(r->d, n, n1, n2, &R, &dt, &kk);
    if (want_robust) {
      /* total internal reflection decides whether a refraction ray is spawned */
      double eta = n1 / n2, ci = -dot(r->d, n);
      double rb = fabs(kk) / (2.0 * eta * eta * fabs(ci) * Ad + s->K * 4 * GAMMA32);
      if (count_robust && rb < out.robust) out.robust = rb;
      if (rb < out.robust_struct) out.robust_struct = rb;
    }
    if (spawn) {
      child_t* c = &out.child[out.n_children++];
      c->r.o = o_up;
      c->r.d = unit(reflect(r->d, n));
      c->r.eo = eo_child;
      c->r.en = en_child;
      c->r.ed = r->ed + 2.0 * An + s->K * 8 * GAMMA32;
      c->w = scl(w, R);
      c->code = code << 1;
      if (has_t) {
        child_t* c2 = &out.child[out.n_children++];
        c2->r.o = sub(ph, scl(n, eps));
        c2->r.d = dt;
        c2->r.eo = eo_child;
        c2->r.en = en_child;
        c2->r.ed = r->ed + 3.0 * An + s->K * 8 * GAMMA32;
        c2->w = scl(w, 1.0 - R);
        c2->code = (code << 1) | 1u;
      }
    }
  }
  return out;
}

/* ------------------------------------------------------------------ */
/* recursive and iterative Whitted tracing                              */
/* ------------------------------------------------------------------ */
typedef struct {
  const orc_scene* s;
  int max_depth, use_bvh;
  uint64_t* counts;     /* 3 + 3 * (max_depth + 1) */
  double robust;
  int want_struct;      /* track robust_struct (every ray, whatever its weight) */
  double robust_struct; /* smallest margin of any decision that changes the pixel's ray counts */
} trace_ctx;

/* The radiance cache's answer for a hit: exp(MLP(encode(p, n, -d))), with
 * n the normal facing the ray; it replaces the hit's local term and all of
 * its children. */
static v3 cache_radiance(const orc_scene* s, const ray_t* r, hit_t h) {
  const prim_t* p = &s->prims[h.prim];
  v3 ph = add(r->o, scl(r->d, h.t));
  v3 ng = geometric_normal(p, ph);
  v3 n = dot(r->d, ng) > 0.0 ? scl(ng, -1.0) : ng;
  double pnv[9] = {0, 0, 0, n.x, n.y, n.z, -r->d.x, -r->d.y, -r->d.z};
  double pc[3] = {ph.x, ph.y, ph.z};
  /* normalised position first, then the encoding of an identity box */
  for (int j = 0; j < 3; ++j) pnv[j] = (pc[j] - s->nrc_lo[j]) * s->nrc_inv_ext[j];
  double f[96], y[3];
  double zero[3] = {0, 0, 0}, one[3] = {1, 1, 1};
  orc_nrc_encode(1, pnv, zero, one, f);
  if (s->nrc_bf16)
    for (int k = 0; k < 96; ++k) f[k] = orc_round_bf16(f[k]);
  orc_mlp_forward_ex(1, f, s->nrc_W, s->nrc_B, y, s->nrc_bf16);
  return mk(y[0], y[1], y[2]);
}

/* Radiance arriving along r at depth `depth`, times the ray weight w.  The
 * path vertex the ray leads to is `code`: 1 for the camera ray, then
 * 2c (reflection) and 2c + 1 (refraction or diffuse bounce) for the
 * children of vertex c, with CODE_BOUNCE set on a diffuse bounce. */
static v3 trace_rec(trace_ctx* cx, const ray_t* r, int depth, v3 w, int64_t pixel, uint32_t code, int32_t* prim0,
                    double* t0) {
  const orc_scene* s = cx->s;
  cx->counts[depth == 0 ? 0 : 2]++;
  cx->counts[3 + 3 * depth + 0]++;
  int want = maxc(w) * s->l_max >= 1e-3;
  hit_t h = closest_hit(s, r, 0.0, cx->use_bvh, want || cx->want_struct);
  if (want && h.robust < cx->robust) cx->robust = h.robust;
  if (cx->want_struct && h.robust < cx->robust_struct) cx->robust_struct = h.robust;
  if (prim0) { *prim0 = h.prim; *t0 = h.t; }
  if (h.prim < 0) return mul(w, s->bg);
  cx->counts[3 + 3 * depth + 2]++;
  if (depth == s->nrc_depth) {
    /* the cache stands for the radiance the hit reflects; its own L_e is
     * added as at any hit (not on a diffuse bounce, whose parent sampled
     * the emitters) */
    v3 c = cache_radiance(s, r, h);
    if (!(code & CODE_BOUNCE)) c = add(c, s->mats[s->prims[h.prim].mat].emis);
    return mul(w, c);
  }
  shade_t sh = shade_hit(s, r, w, h.prim, h.t, h.cosn, depth < cx->max_depth, cx->use_bvh, 1, pixel, code);
  if (sh.robust < cx->robust) cx->robust = sh.robust;
  if (sh.robust_struct < cx->robust_struct) cx->robust_struct = sh.robust_struct;
  cx->counts[1] += (uint64_t)sh.n_shadow;
  cx->counts[3 + 3 * depth + 1] += (uint64_t)sh.n_shadow;
  v3 c = sh.local;
  for (int k = 0; k < sh.n_children; ++k)
    c = add(c, trace_rec(cx, &sh.child[k].r, depth + 1, sh.child[k].w, pixel, sh.child[k].code, NULL, NULL));
  return c;
}

/* The iteration-over-depth form (Sec. IV.A): all rays of one depth are
 * processed before the next; every contribution carries its explicit
 * weight.  Same arithmetic as trace_rec, accumulated in another order. */
typedef struct { ray_t r; v3 w; uint32_t code; } qray;
static v3 trace_iter(trace_ctx* cx, const ray_t* r0, int64_t pixel, int32_t* prim0, double* t0) {
  const orc_scene* s = cx->s;
  int cap = 1 << (cx->max_depth + 2);
  qray* cur = (qray*)malloc(sizeof(qray) * (size_t)cap);
  qray* nxt = (qray*)malloc(sizeof(qray) * (size_t)cap);
  int ncur = 1, nnxt;
  cur[0].r = *r0; cur[0].w = mk(1, 1, 1); cur[0].code = 1u;
  v3 pix = mk(0, 0, 0);
  for (int depth = 0; depth <= cx->max_depth && ncur > 0; ++depth) {
    nnxt = 0;
    for (int i = 0; i < ncur; ++i) {
      cx->counts[depth == 0 ? 0 : 2]++;
      cx->counts[3 + 3 * depth + 0]++;
      hit_t h = closest_hit(s, &cur[i].r, 0.0, 0, 0);
      if (depth == 0 && prim0) { *prim0 = h.prim; *t0 = h.t; }
      if (h.prim < 0) { pix = add(pix, mul(cur[i].w, s->bg)); continue; }
      cx->counts[3 + 3 * depth + 2]++;
      if (depth == s->nrc_depth) {
        v3 c = cache_radiance(s, &cur[i].r, h);
        if (!(cur[i].code & CODE_BOUNCE)) c = add(c, s->mats[s->prims[h.prim].mat].emis);
        pix = add(pix, mul(cur[i].w, c));
        continue;
      }
      shade_t sh = shade_hit(s, &cur[i].r, cur[i].w, h.prim, h.t, h.cosn, depth < cx->max_depth, 0, 0, pixel,
                             cur[i].code);
      cx->counts[1] += (uint64_t)sh.n_shadow;
      cx->counts[3 + 3 * depth + 1] += (uint64_t)sh.n_shadow;
      pix = add(pix, sh.local);
      for (int k = 0; k < sh.n_children; ++k) {
        nxt[nnxt].r = sh.child[k].r;
        nxt[nnxt].w = sh.child[k].w;
        nxt[nnxt].code = sh.child[k].code;
        nnxt++;
      }
    }
    qray* tmp = cur; cur = nxt; nxt = tmp;
    ncur = nnxt;
  }
  free(cur);
  free(nxt);
  return pix;
}

/* ------------------------------------------------------------------ */
/* camera (the paper gives none): pinhole, vertical field of view,       */
/* pixel centres at +0.5, row 0 at the top.                              */
/* ------------------------------------------------------------------ */
/* The ray through image point (px, py) in pixel units (the centre of pixel
 * (x, y) is (x + 0.5, y + 0.5)). */
static void camera_ray_at(const in_cam* cam, int W, int H, double px, double py, v3* o, v3* d) {
  v3 eye = f3(cam->eye), at = f3(cam->look_at), up = f3(cam->up);
  v3 f = unit(sub(at, eye));
  v3 r = unit(cross(f, up));
  v3 u = cross(r, f);
  double h = tan(0.5 * (double)cam->vfov_deg * M_PI / 180.0);
  double a = (double)W / (double)H;
  double sx = (2.0 * px / W - 1.0) * h * a;
  double ty = (1.0 - 2.0 * py / H) * h;
  *o = eye;
  *d = unit(add(f, add(scl(r, sx), scl(u, ty))));
}

static void camera_ray(const in_cam* cam, int W, int H, int x, int y, v3* o, v3* d) {
  camera_ray_at(cam, W, H, x + 0.5, y + 0.5, o, d);
}

void orc_camera_ray(const void* cam, int width, int height, int x, int y, double* o, double* d) {
  v3 oo, dd;
  camera_ray((const in_cam*)cam, width, height, x, y, &oo, &dd);
  o[0] = oo.x; o[1] = oo.y; o[2] = oo.z;
  d[0] = dd.x; d[1] = dd.y; d[2] = dd.z;
}

/* ------------------------------------------------------------------ */
/* scene                                                                */
/* ------------------------------------------------------------------ */
static int finite3(const float* p) { return isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]); }

orc_scene* orc_scene_create(const void* spheres, int64_t ns, const void* triangles, int64_t nt,
                            const void* materials, int64_t nm, const void* lights, int64_t nl,
                            const double* background, double eps_scale, double fragile_k) {
  if (ns < 0 || nt < 0 || nm <= 0 || nl < 0) return NULL;
  orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
  s->n_spheres = ns;
  s->n_prims = ns + nt;
  s->prims = (prim_t*)calloc((size_t)(s->n_prims > 0 ? s->n_prims : 1), sizeof(prim_t));
  s->n_mats = nm;
  s->mats = (mat_t*)calloc((size_t)nm, sizeof(mat_t));
  s->n_lights = nl;
  s->lights = (light_t*)calloc((size_t)(nl > 0 ? nl : 1), sizeof(light_t));
  s->bg = mk(background[0], background[1], background[2]);
  s->eps_scale = eps_scale;
  s->K = fragile_k;
  s->nrc_depth = -1;
  s->strata = 1;
  const in_mat* im = (const in_mat*)materials;
  double ks_max = 0, em_max = 0;
  for (int64_t i = 0; i < nm; ++i) {
    mat_t* m = &s->mats[i];
    m->kind = im[i].kind;
    m->albedo = f3(im[i].albedo);
    m->ks = im[i].ks;
    m->shin = im[i].shininess;
    m->refl = im[i].reflectivity;
    m->ior = im[i].ior;
    m->emis = f3(im[i].emission);
    if (m->ks > ks_max) ks_max = m->ks;
    if (maxc(m->emis) > em_max) em_max = maxc(m->emis);
  }
  const in_light* il = (const in_light*)lights;
  double lsum = 0;
  for (int64_t i = 0; i < nl; ++i) {
    s->lights[i].pos = f3(il[i].pos);
    s->lights[i].inten = f3(il[i].intensity);
    lsum += maxc(s->lights[i].inten);
  }
  s->l_max = maxc(s->bg) + lsum * (1.0 + ks_max) + em_max;
  const in_sphere* is = (const in_sphere*)spheres;
  const in_tri* it = (const in_tri*)triangles;
  v3 slo = mk(INFINITY, INFINITY, INFINITY), shi = mk(-INFINITY, -INFINITY, -INFINITY);
  for (int64_t i = 0; i < ns; ++i) {
    prim_t* p = &s->prims[i];
    if (!finite3(is[i].c) || !isfinite(is[i].r) || !(is[i].r > 0) || is[i].mat >= (uint32_t)nm) goto bad;
    p->is_sphere = 1;
    p->mat = is[i].mat;
    p->c = f3(is[i].c);
    p->r = is[i].r;
    p->lo = sub(p->c, mk(p->r, p->r, p->r));
    p->hi = add(p->c, mk(p->r, p->r, p->r));
    p->centroid = p->c;
    p->scale = maxabs(p->c) + p->r;
    p->aspect = 1.0;
    p->bc = p->c;
    p->brad = p->r;
  }
  for (int64_t j = 0; j < nt; ++j) {
    prim_t* p = &s->prims[ns + j];
    if (!finite3(it[j].v0) || !finite3(it[j].v1) || !finite3(it[j].v2) || it[j].mat >= (uint32_t)nm) goto bad;
    p->is_sphere = 0;
    p->mat = it[j].mat;
    p->v0 = f3(it[j].v0); p->v1 = f3(it[j].v1); p->v2 = f3(it[j].v2);
    p->lo = vmin(p->v0, vmin(p->v1, p->v2));
    p->hi = vmax(p->v0, vmax(p->v1, p->v2));
    p->centroid = scl(add(p->v0, add(p->v1, p->v2)), 1.0 / 3.0);
    p->scale = fmax(maxabs(p->v0), fmax(maxabs(p->v1), maxabs(p->v2)));
    double area2 = len(cross(sub(p->v1, p->v0), sub(p->v2, p->v0)));
    double emax = fmax(len(sub(p->v1, p->v0)), fmax(len(sub(p->v2, p->v0)), len(sub(p->v2, p->v1))));
    double h_min = emax > 0 ? area2 / emax : 0;
    p->aspect = h_min > 0 ? emax / h_min : 1e30;
    p->bc = p->centroid;
    p->brad = fmax(len(sub(p->v0, p->bc)), fmax(len(sub(p->v1, p->bc)), len(sub(p->v2, p->bc))));
  }
  /* emissive primitives, in id order */
  s->emitters = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s->n_prims > 0 ? s->n_prims : 1));
  s->n_emitters = 0;
  for (int64_t i = 0; i < s->n_prims; ++i)
    if (maxc(s->mats[s->prims[i].mat].emis) > 0.0) s->emitters[s->n_emitters++] = i;
  if (s->n_emitters > 0) s->l_max = INFINITY;
  for (int64_t i = 0; i < s->n_prims; ++i) {
    slo = vmin(slo, s->prims[i].lo);
    shi = vmax(shi, s->prims[i].hi);
  }
  if (s->n_prims == 0) { slo = mk(0, 0, 0); shi = mk(0, 0, 0); }
  s->scene_lo = slo;
  s->scene_hi = shi;
  if (s->n_prims > 0) {
    s->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)s->n_prims);
    for (int64_t i = 0; i < s->n_prims; ++i) s->order[i] = i;
    s->nodes = (node_t*)calloc((size_t)(2 * s->n_prims), sizeof(node_t));
    s->n_nodes = 0;
    bvh_build_rec(s, 0, s->n_prims);
  }
  return s;
bad:
  orc_scene_free(s);
  return NULL;
}

void orc_scene_free(orc_scene* s) {
  if (!s) return;
  free(s->prims); free(s->mats); free(s->lights); free(s->alights); free(s->emitters); free(s->nodes);
  free(s->order);
  free(s->nrc_W); free(s->nrc_B);
  free(s);
}

int64_t orc_bvh_node_count(const orc_scene* s) { return s->n_nodes; }

int orc_set_area_lights(orc_scene* s, const void* lights, int64_t n) {
  if (!s || n < 0 || (n > 0 && !lights)) return 1;
  const in_alight* il = (const in_alight*)lights;
  alight_t* a = (alight_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(alight_t));
  for (int64_t i = 0; i < n; ++i) {
    if (!finite3(il[i].corner) || !finite3(il[i].edge_u) || !finite3(il[i].edge_v) || !finite3(il[i].radiance)) {
      free(a);
      return 1;
    }
    a[i].corner = f3(il[i].corner);
    a[i].eu = f3(il[i].edge_u);
    a[i].ev = f3(il[i].edge_v);
    a[i].L = f3(il[i].radiance);
    v3 c = cross(a[i].eu, a[i].ev);
    a[i].area = len(c);
    if (!(a[i].area > 0.0)) {
      free(a);
      return 1;
    }
    a[i].nl = scl(c, 1.0 / a[i].area);
  }
  free(s->alights);
  s->alights = a;
  s->n_alights = n;
  /* a sampled area light has no small bound: track every decision */
  if (n > 0) s->l_max = INFINITY;
  return 0;
}

void orc_set_pass(orc_scene* s, uint64_t seed, int32_t pass, int32_t strata, int32_t jitter) {
  s->seed_lo = (uint32_t)seed;
  s->seed_hi = (uint32_t)(seed >> 32);
  s->pass = pass;
  s->strata = strata > 0 ? strata : 1;
  s->jitter = jitter != 0;
}

void orc_set_diffuse_bounce(orc_scene* s, int32_t on) { s->bounce = on != 0; }

void orc_set_cache(orc_scene* s, int depth, const double* W, const double* B, int bf16, const double* lo,
                   const double* inv_ext) {
  free(s->nrc_W);
  free(s->nrc_B);
  s->nrc_W = s->nrc_B = NULL;
  s->nrc_depth = depth;
  if (depth < 0) return;
  s->nrc_W = (double*)malloc(sizeof(double) * ORC_NRC_NW);
  s->nrc_B = (double*)malloc(sizeof(double) * ORC_NRC_NB);
  memcpy(s->nrc_W, W, sizeof(double) * ORC_NRC_NW);
  memcpy(s->nrc_B, B, sizeof(double) * ORC_NRC_NB);
  s->nrc_bf16 = bf16;
  for (int j = 0; j < 3; ++j) {
    s->nrc_lo[j] = lo[j];
    s->nrc_inv_ext[j] = inv_ext[j];
  }
}

/* ------------------------------------------------------------------ */
/* entry points                                                         */
/* ------------------------------------------------------------------ */
int orc_render(const orc_scene* s, const void* cam, int W, int H, int max_depth, int mode,
               const int64_t* pixels, int64_t n_pixels, double* rgb, int32_t* prim, double* t,
               double* robust, uint64_t* counts, int nthreads) {
  return orc_render_px(s, cam, W, H, max_depth, mode, pixels, n_pixels, rgb, prim, t, robust, counts, NULL, NULL,
                       nthreads);
}

int orc_render_px(const orc_scene* s, const void* cam, int W, int H, int max_depth, int mode,
                  const int64_t* pixels, int64_t n_pixels, double* rgb, int32_t* prim, double* t,
                  double* robust, uint64_t* counts, double* robust_struct, uint32_t* px_counts, int nthreads) {
  if (!s || !cam || W < 1 || H < 1 || max_depth < 0 || max_depth > MAX_DEPTH_LIMIT) return 1;
  if (robust_struct && mode == 2) return 1;   /* the iterative form tracks no margins */
  int64_t n = pixels ? n_pixels : (int64_t)W * H;
  int nc = 3 + 3 * (max_depth + 1);
  uint64_t* total = (uint64_t*)calloc((size_t)nc, sizeof(uint64_t));
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
  {
    uint64_t* cnt = (uint64_t*)calloc((size_t)nc, sizeof(uint64_t));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
    for (int64_t i = 0; i < n; ++i) {
      int64_t pix = pixels ? pixels[i] : i;
      int x = (int)(pix % W), y = (int)(pix / W);
      ray_t r;
      double jx = 0.5, jy = 0.5;   /* the pixel centre, or the pass's point inside the pixel */
      if (s->jitter) pass_sample(s, pix, 0u, SLOT_PIXEL, &jx, &jy);
      camera_ray_at((const in_cam*)cam, W, H, x + jx, y + jy, &r.o, &r.d);
      r.eo = 0.0;
      r.en = 0.0;
      r.ed = s->K * 4 * GAMMA32;
      trace_ctx cx;
      cx.s = s; cx.max_depth = max_depth; cx.use_bvh = (mode == 1); cx.counts = cnt;
      cx.robust = ROBUST_CAP;
      cx.want_struct = robust_struct != NULL;
      cx.robust_struct = ROBUST_CAP;
      /* per-pixel counts: this pixel's share of the per-depth totals */
      uint64_t before[2 * (MAX_DEPTH_LIMIT + 1)];
      if (px_counts)
        for (int d = 0; d <= max_depth; ++d) {
          before[2 * d] = cnt[3 + 3 * d];
          before[2 * d + 1] = cnt[3 + 3 * d + 1];
        }
      int32_t p0 = -1;
      double t0 = INFINITY;
      v3 c;
      if (mode == 2) c = trace_iter(&cx, &r, pix, &p0, &t0);
      else c = trace_rec(&cx, &r, 0, mk(1, 1, 1), pix, 1u, &p0, &t0);
      if (rgb) { rgb[3 * i] = c.x; rgb[3 * i + 1] = c.y; rgb[3 * i + 2] = c.z; }
      if (prim) prim[i] = p0;
      if (t) t[i] = p0 >= 0 ? t0 : INFINITY;
      if (robust) robust[i] = cx.robust;
      if (robust_struct) robust_struct[i] = cx.robust_struct;
      if (px_counts)
        for (int d = 0; d <= max_depth; ++d) {
          px_counts[(size_t)i * 2 * (max_depth + 1) + 2 * d] = (uint32_t)(cnt[3 + 3 * d] - before[2 * d]);
          px_counts[(size_t)i * 2 * (max_depth + 1) + 2 * d + 1] =
              (uint32_t)(cnt[3 + 3 * d + 1] - before[2 * d + 1]);
        }
    }
#ifdef _OPENMP
#pragma omp critical
#endif
    for (int k = 0; k < nc; ++k) total[k] += cnt[k];
    free(cnt);
  }
  if (counts) memcpy(counts, total, sizeof(uint64_t) * (size_t)nc);
  free(total);
  return 0;
}

int orc_closest_hits(const orc_scene* s, int64_t n, const float* o, const float* d, double tmin,
                     int use_bvh, int32_t* prim, double* t, double* robust, int nthreads) {
  if (!s) return 1;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
#endif
  for (int64_t i = 0; i < n; ++i) {
    ray_t r;
    r.o = f3(o + 3 * i);
    r.d = f3(d + 3 * i);
    r.eo = 0; r.ed = 0; r.en = 0;
    hit_t h = closest_hit(s, &r, tmin, use_bvh, robust != NULL);
    prim[i] = h.prim;
    t[i] = h.prim >= 0 ? h.t : INFINITY;
    if (robust) robust[i] = h.robust;
  }
  return 0;
}

int orc_any_hits(const orc_scene* s, int64_t n, const float* o, const float* d, double tmin,
                 const float* tmax, int use_bvh, uint8_t* occluded, double* robust, int nthreads) {
  if (!s) return 1;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
#endif
  for (int64_t i = 0; i < n; ++i) {
    ray_t r;
    r.o = f3(o + 3 * i);
    r.d = f3(d + 3 * i);
    r.eo = 0; r.ed = 0; r.en = 0;
    double rb = ROBUST_CAP;
    occluded[i] = (uint8_t)any_hit(s, &r, tmin, tmax[i], use_bvh, robust ? &rb : NULL);
    if (robust) robust[i] = rb;
  }
  return 0;
}

int orc_sphere_roots(const double* o, const double* d, const double* c, double r, double* t) {
  v3 f = sub(mk(o[0], o[1], o[2]), mk(c[0], c[1], c[2]));
  v3 dd = mk(d[0], d[1], d[2]);
  double a = dot(dd, dd), b = 2.0 * dot(f, dd), cc = dot(f, f) - r * r;
  double disc = b * b - 4.0 * a * cc;
  if (disc < 0) return 0;
  double sq = sqrt(disc);
  t[0] = (-b - sq) / (2.0 * a);
  t[1] = (-b + sq) / (2.0 * a);
  return disc == 0.0 ? 1 : 2;
}

int orc_triangle_hit(const double* o, const double* d, const double* v0, const double* v1,
                     const double* v2, double* t, double* u, double* v) {
  prim_t p;
  memset(&p, 0, sizeof p);
  p.v0 = mk(v0[0], v0[1], v0[2]);
  p.v1 = mk(v1[0], v1[1], v1[2]);
  p.v2 = mk(v2[0], v2[1], v2[2]);
  v3 oo = mk(o[0], o[1], o[2]), dd = mk(d[0], d[1], d[2]);
  cand_t c = tri_cand(&p, oo, dd, 0.0);
  v3 e1 = sub(p.v1, p.v0), e2 = sub(p.v2, p.v0);
  v3 P = cross(dd, e2);
  double det = dot(e1, P);
  if (det != 0) {
    v3 T = sub(oo, p.v0);
    *u = dot(T, P) / det;
    *v = dot(dd, cross(T, e1)) / det;
  }
  *t = c.t;
  return c.hit;
}

int orc_refract(const double* d, const double* n, double n1, double n2, double* R, double* dt) {
  v3 o;
  int ok = refract_schlick(mk(d[0], d[1], d[2]), mk(n[0], n[1], n[2]), n1, n2, R, &o, NULL);
  if (ok) { dt[0] = o.x; dt[1] = o.y; dt[2] = o.z; }
  return ok;
}
