/*
 * pft_oracle.c -- FP64 CPU oracle for the direct Fourier transform of polygonal
 * areas and closed surfaces of triangles or planar polygons (B. B. Maranville,
 * arXiv 2104.08309).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, double-precision
 * statement of what the CUDA library computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load it; the library itself never
 * does, and the two share no code.
 *
 * Convention (Sec. 2, Eq. 7): FT(Q) = integral over the region of exp(+i Q.r),
 * with no 2 pi in the exponent.  Loops are counter-clockwise for positive area;
 * triangles are counter-clockwise seen from outside (outward normal).
 *
 * Every routine loops over Q and over segments/faces one by one, in FP64, with
 * Neumaier-compensated sums.  Limits the paper's formulas leave undefined
 * (Q = 0, sinc(0), Q parallel to a face normal, |Q| -> 0) take explicit
 * branches, each a closed form or a convergent series of the same integral.
 *
 * Parity of every function here is pinned by the tests against closed forms
 * (rectangle, prism, disc, sphere), brute-force quadrature, invariances and
 * finite differences; none is "parity unpinned".
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KMAX 48            /* terms of the simplex series (ample below |nodes| = 4) */
#define TAU_SINC 1e-3      /* |u| below which sinc uses its Taylor polynomial       */
#define TAU_FACE 1e-2      /* face phase spread below which the face series is used */
#define TAU_Q 0.5          /* |Q| * max|r| below which the whole-shape series is used */
#define TAU_GRAD 4.0       /* spread above which a triangle is subdivided (gradient)  */

/* ---------------------------------------------------------------------------
 * Small helpers.
 * ------------------------------------------------------------------------- */

typedef struct { double re, im, cre, cim; } csum_t;   /* Neumaier complex sum */

static void nsum(double* s, double* c, double x) {
  double t = *s + x;
  if (fabs(*s) >= fabs(x)) *c += (*s - t) + x; else *c += (x - t) + *s;
  *s = t;
}
static void csum_add(csum_t* a, double complex z) { nsum(&a->re, &a->cre, creal(z)); nsum(&a->im, &a->cim, cimag(z)); }
static double complex csum_get(const csum_t* a) { return (a->re + a->cre) + I * (a->im + a->cim); }

static double inv_fact[KMAX + 8];
static int inv_fact_ready = 0;
static void init_tables(void) {
  if (inv_fact_ready) return;
  double f = 1.0;
  inv_fact[0] = 1.0;
  for (int k = 1; k < KMAX + 8; ++k) { f *= (double)k; inv_fact[k] = 1.0 / f; }
  inv_fact_ready = 1;
}

/* sinc(u) = sin(u)/u, unnormalised, as in the midpoint form of Eq. 6 (Sec. 2). */
static double sinc(double u) {
  if (fabs(u) < TAU_SINC) { double u2 = u * u; return 1.0 - u2 / 6.0 * (1.0 - u2 / 20.0 * (1.0 - u2 / 42.0)); }
  return sin(u) / u;
}

/* Complete homogeneous symmetric polynomials h_0..h_K of the n nodes x. */
static void homog(const double* x, int n, double* h, int K) {
  h[0] = 1.0;
  for (int k = 1; k <= K; ++k) h[k] = 0.0;
  for (int j = 0; j < n; ++j)
    for (int k = 1; k <= K; ++k) h[k] += x[j] * h[k - 1];
}

/*
 * Simplex series: sum_k i^k h_k(x) / (k+p)!.
 * For the n nodes x_j = Q.r_j of an (n-1)-simplex, the integral of exp(iQ.r)
 * over the simplex is (n-1)! * |simplex| * (this series with p = n-1): the
 * Taylor expansion of exp(iQ.r) integrated term by term with the simplex
 * moment formula.  Used for the limits the paper's sums cannot reach.
 */
static double complex simplex_series(const double* x, int n, int p) {
  double h[KMAX + 1];
  homog(x, n, h, KMAX);
  double re = 0.0, im = 0.0;
  for (int k = KMAX; k >= 0; --k) {           /* smallest terms first */
    double t = h[k] * inv_fact[k + p];
    switch (k & 3) { case 0: re += t; break; case 1: im += t; break; case 2: re -= t; break; default: im -= t; }
  }
  return re + I * im;
}

/* ---------------------------------------------------------------------------
 * 2D: region bounded by closed loops of vertices (CSR: loop l is
 * verts[loop_off[l] .. loop_off[l+1]-1], the last vertex joined to the first).
 * ------------------------------------------------------------------------- */

/* Signed shoelace area: the Q = 0 value of FT_A. */
static double area2d(const double* v, const int64_t* off, int64_t nl) {
  double s = 0.0, c = 0.0;
  for (int64_t l = 0; l < nl; ++l)
    for (int64_t j = off[l]; j < off[l + 1]; ++j) {
      int64_t k = (j + 1 < off[l + 1]) ? j + 1 : off[l];
      nsum(&s, &c, 0.5 * (v[2 * j] * v[2 * k + 1] - v[2 * k] * v[2 * j + 1]));
    }
  return s + c;
}

/*
 * Segment term of Eq. 6 (Sec. 2): for p0 -> p1, Delta = p1 - p0,
 *   T = -i (Qx Dy - Qy Dx) exp(iQ.(p0+p1)/2) sinc(Q.Delta/2)      (times 1/|Q|^2)
 * which equals the exponential-difference form of Eq. 4 segment by segment.
 * Returned without the 1/|Q|^2 factor.
 */
static double complex seg_term(double qx, double qy, double x0, double y0, double x1, double y1) {
  double dx = x1 - x0, dy = y1 - y0;
  double w = qx * dy - qy * dx;
  double u = 0.5 * (qx * dx + qy * dy);
  double phi = 0.5 * (qx * (x0 + x1) + qy * (y0 + y1));
  return -I * w * sinc(u) * cexp(I * phi);
}

static double complex ft2d_at(const double* v, const int64_t* off, int64_t nl,
                              double qx, double qy, double rmax, double area) {
  double q2 = qx * qx + qy * qy;
  if (q2 == 0.0) return area;                  /* Q = 0: the area itself */
  csum_t acc = {0, 0, 0, 0};
  if (sqrt(q2) * rmax < TAU_Q) {
    /* |Q| -> 0: the segment sum cancels to O(|Q|^2); integrate instead over the
       fan of triangles (origin, p_j, p_{j+1}) with the simplex series. */
    for (int64_t l = 0; l < nl; ++l)
      for (int64_t j = off[l]; j < off[l + 1]; ++j) {
        int64_t k = (j + 1 < off[l + 1]) ? j + 1 : off[l];
        double a2 = v[2 * j] * v[2 * k + 1] - v[2 * k] * v[2 * j + 1];   /* twice the signed area */
        double x[2] = {qx * v[2 * j] + qy * v[2 * j + 1], qx * v[2 * k] + qy * v[2 * k + 1]};
        csum_add(&acc, a2 * simplex_series(x, 2, 2));
      }
    return csum_get(&acc);
  }
  for (int64_t l = 0; l < nl; ++l)
    for (int64_t j = off[l]; j < off[l + 1]; ++j) {
      int64_t k = (j + 1 < off[l + 1]) ? j + 1 : off[l];
      csum_add(&acc, seg_term(qx, qy, v[2 * j], v[2 * j + 1], v[2 * k], v[2 * k + 1]));
    }
  return csum_get(&acc) / q2;
}

static double rmax2d(const double* v, int64_t n) {
  double r = 0.0;
  for (int64_t j = 0; j < n; ++j) r = fmax(r, hypot(v[2 * j], v[2 * j + 1]));
  return r;
}

/* FT_A of the region bounded by all loops, at each of the n_q points q[n_q][2]. */
int orc_ft2d(const double* verts, const int64_t* loop_off, int64_t n_loops,
             const double* q, int64_t n_q, double* out, int n_threads) {
  init_tables();
  int64_t nv = loop_off[n_loops];
  double rmax = rmax2d(verts, nv), area = area2d(verts, loop_off, n_loops);
#pragma omp parallel for schedule(dynamic, 16) num_threads(n_threads)
  for (int64_t iq = 0; iq < n_q; ++iq) {
    double complex f = ft2d_at(verts, loop_off, n_loops, q[2 * iq], q[2 * iq + 1], rmax, area);
    out[2 * iq] = creal(f); out[2 * iq + 1] = cimag(f);
  }
  return 0;
}

/* Per-segment terms of Eq. 4/6 (with the 1/|Q|^2 factor) at one Q; out[n_seg][2]. */
int orc_seg_terms2d(const double* verts, const int64_t* loop_off, int64_t n_loops,
                    double qx, double qy, double* out) {
  double q2 = qx * qx + qy * qy;
  for (int64_t l = 0; l < n_loops; ++l)
    for (int64_t j = loop_off[l]; j < loop_off[l + 1]; ++j) {
      int64_t k = (j + 1 < loop_off[l + 1]) ? j + 1 : loop_off[l];
      double complex t = seg_term(qx, qy, verts[2 * j], verts[2 * j + 1], verts[2 * k], verts[2 * k + 1]) / q2;
      out[2 * j] = creal(t); out[2 * j + 1] = cimag(t);
    }
  return 0;
}

/*
 * Batched 2D: polygon i is verts[poly_off[i] .. poly_off[i+1]-1]; it is
 * evaluated on q[q_off[i] .. q_off[i+1]-1] (or on all n_q points when q_off is
 * NULL); results are packed in the same order.
 */
int orc_ft2d_batched(const double* verts, const int64_t* poly_off, int64_t n_polys,
                     const double* q, const int64_t* q_off, int64_t n_q, double* out, int n_threads) {
  init_tables();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
  for (int64_t i = 0; i < n_polys; ++i) {
    int64_t lo[2] = {0, poly_off[i + 1] - poly_off[i]};
    const double* v = verts + 2 * poly_off[i];
    double rmax = rmax2d(v, lo[1]), area = area2d(v, lo, 1);
    int64_t q0 = q_off ? q_off[i] : 0, q1 = q_off ? q_off[i + 1] : n_q;
    int64_t o0 = q_off ? q_off[i] : i * n_q;
    for (int64_t iq = q0; iq < q1; ++iq) {
      double complex f = ft2d_at(v, lo, 1, q[2 * iq], q[2 * iq + 1], rmax, area);
      out[2 * (o0 + iq - q0)] = creal(f); out[2 * (o0 + iq - q0) + 1] = cimag(f);
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * 3D: closed surface of triangles faces[n_f][3] (0-based into verts[n_v][3]).
 * ------------------------------------------------------------------------- */

static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1]; c[1] = a[2] * b[0] - a[0] * b[2]; c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/*
 * One face's term I_m of Eq. 14 with the sign fixed (Sec. 3, Eqs. 11-14).
 * With N = (p1-p0) x (p2-p0) (|N| = 2 area, along the outward normal),
 * s = Q.N, X = N x Q (|X| = |N| |Q_perp|), d_l = p_{l+1} - p_l (wrapping):
 *   I_m = -s / (|Q|^2 |X|^2) * sum_l Q.(d_l x N) exp(iQ.(p_l+p_{l+1})/2) sinc(Q.d_l/2)
 * which is Eq. 13 (face factor -i Q_par/Q^2 exp(i Q_par r_par) times the in-plane
 * 2D transform) with the in-plane transform taken from Eq. 6.  As printed, Eq. 14
 * has the opposite overall sign; this sign reproduces the prism face values of
 * Sec. 4.2 and gives FT(0) = +volume for outward faces.
 *
 * When the face's phase spread max_l |Q.d_l| is below TAU_FACE the edge sum
 * cancels (it is O(|Q_perp| L) relative to its terms) and is undefined for
 * Q parallel to N; there Eq. 13 is evaluated directly, the in-face integral of
 * exp(iQ.r) coming from the simplex series:  I_m = -i s exp(i mu) G(a) / |Q|^2,
 * mu = mean_k Q.p_k, a_k = Q.p_k - mu, G = sum_k i^k h_k(a)/(k+2)!.
 * Returned without the 1/|Q|^2 factor.
 */
static double complex face_term(const double* Q, const double* p0, const double* p1, const double* p2) {
  const double* p[3] = {p0, p1, p2};
  double e1[3], e2[3], N[3], X[3];
  for (int c = 0; c < 3; ++c) { e1[c] = p1[c] - p0[c]; e2[c] = p2[c] - p0[c]; }
  cross3(e1, e2, N);
  if (N[0] == 0.0 && N[1] == 0.0 && N[2] == 0.0) return 0.0;   /* degenerate face: no area */
  double s = dot3(Q, N);
  cross3(N, Q, X);
  double x2 = dot3(X, X);
  double alpha[3] = {dot3(Q, p0), dot3(Q, p1), dot3(Q, p2)};
  double spread = 0.0;
  for (int l = 0; l < 3; ++l) {
    double dl[3];
    for (int c = 0; c < 3; ++c) dl[c] = p[(l + 1) % 3][c] - p[l][c];
    spread = fmax(spread, fabs(dot3(Q, dl)));
  }
  if (spread < TAU_FACE || x2 == 0.0) {
    double mu = (alpha[0] + alpha[1] + alpha[2]) / 3.0;
    double a[3] = {alpha[0] - mu, alpha[1] - mu, alpha[2] - mu};
    return -I * s * cexp(I * mu) * simplex_series(a, 3, 2);
  }
  csum_t acc = {0, 0, 0, 0};
  for (int l = 0; l < 3; ++l) {
    const double* a = p[l];
    const double* b = p[(l + 1) % 3];
    double dl[3], t[3], m[3];
    for (int c = 0; c < 3; ++c) { dl[c] = b[c] - a[c]; m[c] = 0.5 * (a[c] + b[c]); }
    cross3(dl, N, t);                                /* in-plane outward edge normal * |d_l| |N| */
    double w = dot3(Q, t);
    double u = 0.5 * dot3(Q, dl);
    csum_add(&acc, w * sinc(u) * cexp(I * dot3(Q, m)));
  }
  return -s / x2 * csum_get(&acc);
}

static double volume3d(const double* v, const int32_t* f, int64_t nf) {
  double s = 0.0, c = 0.0;
  for (int64_t m = 0; m < nf; ++m) {
    const double *a = v + 3 * f[3 * m], *b = v + 3 * f[3 * m + 1], *d = v + 3 * f[3 * m + 2];
    double bxd[3];
    cross3(b, d, bxd);
    nsum(&s, &c, dot3(a, bxd) / 6.0);
  }
  return s + c;
}

static double rmax3d(const double* v, int64_t nv) {
  double r = 0.0;
  for (int64_t j = 0; j < nv; ++j) r = fmax(r, sqrt(dot3(v + 3 * j, v + 3 * j)));
  return r;
}

static double complex ft3d_at(const double* v, const int32_t* f, int64_t nf, const double* Q,
                              double rmax, double vol) {
  double q2 = dot3(Q, Q);
  if (q2 == 0.0) return vol;                    /* Q = 0: the volume itself */
  csum_t acc = {0, 0, 0, 0};
  if (sqrt(q2) * rmax < TAU_Q) {
    /* |Q| -> 0: the face sum cancels to O(|Q|^2); integrate instead over the
       signed tetrahedra (origin, p0, p1, p2) with the simplex series. */
    for (int64_t m = 0; m < nf; ++m) {
      const double *a = v + 3 * f[3 * m], *b = v + 3 * f[3 * m + 1], *d = v + 3 * f[3 * m + 2];
      double bxd[3];
      cross3(b, d, bxd);
      double x[3] = {dot3(Q, a), dot3(Q, b), dot3(Q, d)};
      csum_add(&acc, dot3(a, bxd) * simplex_series(x, 3, 3));
    }
    return csum_get(&acc);
  }
  for (int64_t m = 0; m < nf; ++m)
    csum_add(&acc, face_term(Q, v + 3 * f[3 * m], v + 3 * f[3 * m + 1], v + 3 * f[3 * m + 2]));
  return csum_get(&acc) / q2;
}

static int check_faces(const int32_t* faces, int64_t n_faces, int64_t n_verts) {
  for (int64_t i = 0; i < 3 * n_faces; ++i)
    if (faces[i] < 0 || faces[i] >= n_verts) return 2;
  return 0;
}

/* FT_V of the closed surface at each of the n_q points q[n_q][3]. */
int orc_ft3d(const double* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
             const double* q, int64_t n_q, double* out, int n_threads) {
  init_tables();
  if (check_faces(faces, n_faces, n_verts)) return 2;
  double rmax = rmax3d(verts, n_verts), vol = volume3d(verts, faces, n_faces);
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
  for (int64_t iq = 0; iq < n_q; ++iq) {
    double complex F = ft3d_at(verts, faces, n_faces, q + 3 * iq, rmax, vol);
    out[2 * iq] = creal(F); out[2 * iq + 1] = cimag(F);
  }
  return 0;
}

/* Per-face terms I_m (with 1/|Q|^2) at one Q, Q != 0; out[n_faces][2]. */
int orc_face_terms3d(const double* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
                     const double* Q, double* out) {
  init_tables();
  if (check_faces(faces, n_faces, n_verts)) return 2;
  double q2 = dot3(Q, Q);
  for (int64_t m = 0; m < n_faces; ++m) {
    double complex t = face_term(Q, verts + 3 * faces[3 * m], verts + 3 * faces[3 * m + 1],
                                 verts + 3 * faces[3 * m + 2]) / q2;
    out[2 * m] = creal(t); out[2 * m + 1] = cimag(t);
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * 3D: closed surface of planar polygon faces, CSR: face m has the vertex
 * indices idx[off[m]] .. idx[off[m+1]-1], counter-clockwise seen from outside.
 * ------------------------------------------------------------------------- */

/*
 * One planar polygon face's term I_m of Eq. 14 (sign fixed as for triangles):
 * the same edge sum over the face's n edges, with the face normal direction
 * N = sum_k p_k x p_{k+1} (Newell's vector; for a planar polygon |N| = 2 area
 * and the formula only uses the direction of N, since it is homogeneous of
 * degree 0 in N).  Where the face's phase spread max_k Q.p_k - min_k Q.p_k is
 * below TAU_FACE, or Q is parallel to N, the edge sum cancels; there the face
 * integral is split into the fan triangles (p_0, p_k, p_{k+1}), which tile the
 * polygon with signed areas (exact by additivity), each taken by face_term.
 * Returned without the 1/|Q|^2 factor.
 */
static double complex poly_face_term(const double* Q, const double* v, const int32_t* idx, int64_t n) {
  double N[3] = {0.0, 0.0, 0.0}, lo = INFINITY, hi = -INFINITY;
  for (int64_t k = 0; k < n; ++k) {
    const double* a = v + 3 * idx[k];
    const double* b = v + 3 * idx[(k + 1) % n];
    double c[3];
    cross3(a, b, c);
    for (int j = 0; j < 3; ++j) N[j] += c[j];
    double ph = dot3(Q, a);
    lo = fmin(lo, ph);
    hi = fmax(hi, ph);
  }
  if (N[0] == 0.0 && N[1] == 0.0 && N[2] == 0.0) return 0.0;   /* no area */
  double s = dot3(Q, N), X[3];
  cross3(N, Q, X);
  double x2 = dot3(X, X);
  if (hi - lo < TAU_FACE || x2 == 0.0) {
    csum_t acc = {0, 0, 0, 0};
    for (int64_t k = 1; k + 1 < n; ++k)
      csum_add(&acc, face_term(Q, v + 3 * idx[0], v + 3 * idx[k], v + 3 * idx[k + 1]));
    return csum_get(&acc);
  }
  csum_t acc = {0, 0, 0, 0};
  for (int64_t l = 0; l < n; ++l) {
    const double* a = v + 3 * idx[l];
    const double* b = v + 3 * idx[(l + 1) % n];
    double dl[3], t[3], m[3];
    for (int c = 0; c < 3; ++c) { dl[c] = b[c] - a[c]; m[c] = 0.5 * (a[c] + b[c]); }
    cross3(dl, N, t);
    csum_add(&acc, dot3(Q, t) * sinc(0.5 * dot3(Q, dl)) * cexp(I * dot3(Q, m)));
  }
  return -s / x2 * csum_get(&acc);
}

static int check_poly_faces(const int32_t* idx, const int64_t* off, int64_t n_faces, int64_t n_verts) {
  if (off[0] != 0) return 8;
  for (int64_t m = 0; m < n_faces; ++m)
    if (off[m + 1] - off[m] < 3) return 8;
  for (int64_t i = 0; i < off[n_faces]; ++i)
    if (idx[i] < 0 || idx[i] >= n_verts) return 2;
  return 0;
}

/* FT_V of the closed surface of planar polygon faces at each of the n_q points q[n_q][3]. */
int orc_ft3d_poly(const double* verts, int64_t n_verts, const int32_t* idx, const int64_t* off, int64_t n_faces,
                  const double* q, int64_t n_q, double* out, int n_threads) {
  init_tables();
  int e = check_poly_faces(idx, off, n_faces, n_verts);
  if (e) return e;
  double rmax = rmax3d(verts, n_verts);
  /* Q = 0: the volume, as the signed tetrahedra (origin, p_0, p_k, p_{k+1}) of the fans */
  double vs = 0.0, vc = 0.0;
  for (int64_t m = 0; m < n_faces; ++m)
    for (int64_t k = off[m] + 1; k + 1 < off[m + 1]; ++k) {
      double bxd[3];
      cross3(verts + 3 * idx[k], verts + 3 * idx[k + 1], bxd);
      nsum(&vs, &vc, dot3(verts + 3 * idx[off[m]], bxd) / 6.0);
    }
  const double vol = vs + vc;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
  for (int64_t iq = 0; iq < n_q; ++iq) {
    const double* Q = q + 3 * iq;
    double q2 = dot3(Q, Q);
    double complex F;
    if (q2 == 0.0) {
      F = vol;
    } else if (sqrt(q2) * rmax < TAU_Q) {
      /* |Q| -> 0: the signed tetrahedra of the fans with the simplex series, as for triangles */
      csum_t acc = {0, 0, 0, 0};
      for (int64_t m = 0; m < n_faces; ++m)
        for (int64_t k = off[m] + 1; k + 1 < off[m + 1]; ++k) {
          const double *a = verts + 3 * idx[off[m]], *b = verts + 3 * idx[k], *d = verts + 3 * idx[k + 1];
          double bxd[3];
          cross3(b, d, bxd);
          double x[3] = {dot3(Q, a), dot3(Q, b), dot3(Q, d)};
          csum_add(&acc, dot3(a, bxd) * simplex_series(x, 3, 3));
        }
      F = csum_get(&acc);
    } else {
      csum_t acc = {0, 0, 0, 0};
      for (int64_t m = 0; m < n_faces; ++m)
        csum_add(&acc, poly_face_term(Q, verts, idx + off[m], off[m + 1] - off[m]));
      F = csum_get(&acc) / q2;
    }
    out[2 * iq] = creal(F); out[2 * iq + 1] = cimag(F);
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Gradients with respect to the vertices (shape derivative).
 *
 * Moving the boundary by a velocity field dr changes the integral of exp(iQ.r)
 * over the region by the flux of exp(iQ.r) dr through the boundary:
 *   dF = oint exp(iQ.r) (dr . n) dS.
 * With dr interpolated linearly between the vertices of each segment/face,
 * dF/dp_k is the boundary integral of exp(iQ.r) times the hat function of p_k,
 * times the unnormalised outward normal.  This is independent of the
 * divergence-theorem sums above.  For a loss L(Re F, Im F) with
 * g_Q = dL/dRe F + i dL/dIm F, the vertex gradient is
 *   dL/dp_k = sum_Q Re(conj(g_Q) dF(Q)/dp_k).
 * ------------------------------------------------------------------------- */

/* J0(d) = int_0^1 exp(i t d) dt, J1(d) = int_0^1 t exp(i t d) dt. */
static void seg_moments(double d, double complex* j0, double complex* j1) {
  if (fabs(d) < 1.0) {
    double complex s0 = 0, s1 = 0, term = 1;    /* term = (i d)^n / n! */
    for (int n = 0; n < 40; ++n) {
      s0 += term / (double)(n + 1);
      s1 += term / (double)(n + 2);
      term *= I * d / (double)(n + 1);
    }
    *j0 = s0; *j1 = s1;
  } else {
    double complex e = cexp(I * d);
    *j0 = (e - 1.0) / (I * d);
    *j1 = e / (I * d) + (e - 1.0) / (d * d);
  }
}

/* dL/dverts for a 2D loop region; grad[n_v][2] is overwritten. */
int orc_grad2d(const double* verts, const int64_t* loop_off, int64_t n_loops,
               const double* q, int64_t n_q, const double* g, double* grad, int n_threads) {
  int64_t nv = loop_off[n_loops];
  /* per segment: contributions to its start (0) and end (1) vertex, summed over Q */
  double* seg = (double*)calloc((size_t)(4 * nv), sizeof(double));
  if (!seg) return 1;
#pragma omp parallel for schedule(dynamic, 8) num_threads(n_threads)
  for (int64_t j = 0; j < nv; ++j) {
    int64_t l = 0;
    while (loop_off[l + 1] <= j) ++l;
    int64_t k = (j + 1 < loop_off[l + 1]) ? j + 1 : loop_off[l];
    double x0 = verts[2 * j], y0 = verts[2 * j + 1], x1 = verts[2 * k], y1 = verts[2 * k + 1];
    double nu[2] = {y1 - y0, -(x1 - x0)};       /* outward normal times segment length */
    double s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    for (int64_t iq = 0; iq < n_q; ++iq) {
      double qx = q[2 * iq], qy = q[2 * iq + 1];
      double a0 = qx * x0 + qy * y0, d = qx * (x1 - x0) + qy * (y1 - y0);
      double complex j0, j1;
      seg_moments(d, &j0, &j1);
      double complex e = cexp(I * a0), gb = conj(g[2 * iq] + I * g[2 * iq + 1]);
      double r0 = creal(gb * e * (j0 - j1)), r1 = creal(gb * e * j1);
      nsum(&s[0], &c[0], r0 * nu[0]); nsum(&s[1], &c[1], r0 * nu[1]);
      nsum(&s[2], &c[2], r1 * nu[0]); nsum(&s[3], &c[3], r1 * nu[1]);
    }
    for (int t = 0; t < 4; ++t) seg[4 * j + t] = s[t] + c[t];
  }
  for (int64_t l = 0; l < n_loops; ++l)
    for (int64_t j = loop_off[l]; j < loop_off[l + 1]; ++j) {
      int64_t jp = (j > loop_off[l]) ? j - 1 : loop_off[l + 1] - 1;   /* segment ending at j */
      grad[2 * j] = seg[4 * j + 0] + seg[4 * jp + 2];
      grad[2 * j + 1] = seg[4 * j + 1] + seg[4 * jp + 3];
    }
  free(seg);
  return 0;
}

/*
 * Integral over the triangle (p0,p1,p2) of lambda_j exp(iQ.r) dA for j = 0,1,2
 * (lambda_j the barycentric hat functions), divided by 2*area, from the nodes
 * alpha_k = Q.p_k.  By the simplex moment formula it equals
 *   exp(i mu) sum_k i^k h_k(a_0, a_1, a_2, a_j) / (k+3)!,  a = alpha - mu,
 * (node j counted twice).  Spreads above TAU_GRAD are split into four
 * sub-triangles through the edge midpoints: the integral is additive and the
 * parent's hat functions are linear on each child.
 */
static void tri_hat_moments(const double* alpha, double complex* out) {
  double mx = fmax(alpha[0], fmax(alpha[1], alpha[2])), mn = fmin(alpha[0], fmin(alpha[1], alpha[2]));
  if (mx - mn > TAU_GRAD) {
    double m01 = 0.5 * (alpha[0] + alpha[1]), m12 = 0.5 * (alpha[1] + alpha[2]), m20 = 0.5 * (alpha[2] + alpha[0]);
    /* children (each 1/4 of the area, weights relative to the parent's 2*area) */
    const double ch[4][3] = {{alpha[0], m01, m20}, {m01, alpha[1], m12}, {m20, m12, alpha[2]}, {m01, m12, m20}};
    /* parent's hat values at the children's corners */
    const double hv[4][3][3] = {
      {{1, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}},
      {{0.5, 0.5, 0}, {0, 1, 0}, {0, 0.5, 0.5}},
      {{0.5, 0, 0.5}, {0, 0.5, 0.5}, {0, 0, 1}},
      {{0.5, 0.5, 0}, {0, 0.5, 0.5}, {0.5, 0, 0.5}}};
    for (int j = 0; j < 3; ++j) out[j] = 0;
    for (int c = 0; c < 4; ++c) {
      double complex sub[3];
      tri_hat_moments(ch[c], sub);
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) out[j] += 0.25 * hv[c][k][j] * sub[k];
    }
    return;
  }
  double mu = (alpha[0] + alpha[1] + alpha[2]) / 3.0;
  double complex e = cexp(I * mu);
  for (int j = 0; j < 3; ++j) {
    double x[4] = {alpha[0] - mu, alpha[1] - mu, alpha[2] - mu, alpha[j] - mu};
    out[j] = e * simplex_series(x, 4, 3);
  }
}

/*
 * dL/dverts for a closed triangle surface; grad[n_v][3] is overwritten.
 * If vsel is not NULL, only the n_sel listed vertices are computed and written
 * to grad[n_sel][3] in that order (faces not touching them are skipped).
 */
int orc_grad3d(const double* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
               const double* q, int64_t n_q, const double* g, const int64_t* vsel, int64_t n_sel,
               double* grad, int n_threads) {
  init_tables();
  if (check_faces(faces, n_faces, n_verts)) return 2;
  char* want = NULL;
  if (vsel) {
    want = (char*)calloc((size_t)n_verts, 1);
    if (!want) return 1;
    for (int64_t i = 0; i < n_sel; ++i) want[vsel[i]] = 1;
  }
  double* corner = (double*)calloc((size_t)(9 * n_faces), sizeof(double));
  if (!corner) { free(want); return 1; }
#pragma omp parallel for schedule(dynamic, 4) num_threads(n_threads)
  for (int64_t m = 0; m < n_faces; ++m) {
    const int32_t* fm = faces + 3 * m;
    if (want && !want[fm[0]] && !want[fm[1]] && !want[fm[2]]) continue;
    const double *p0 = verts + 3 * fm[0], *p1 = verts + 3 * fm[1], *p2 = verts + 3 * fm[2];
    double e1[3], e2[3], N[3];
    for (int c = 0; c < 3; ++c) { e1[c] = p1[c] - p0[c]; e2[c] = p2[c] - p0[c]; }
    cross3(e1, e2, N);                     /* outward normal * 2 area */
    double s[3] = {0, 0, 0}, cc[3] = {0, 0, 0};
    for (int64_t iq = 0; iq < n_q; ++iq) {
      const double* Q = q + 3 * iq;
      double alpha[3] = {dot3(Q, p0), dot3(Q, p1), dot3(Q, p2)};
      double complex hm[3];
      tri_hat_moments(alpha, hm);
      /* dF/dp_j = n_hat * (integral of lambda_j exp(iQ.r) dA) = N * hm[j]  (|N| = 2 area) */
      double complex gb = conj(g[2 * iq] + I * g[2 * iq + 1]);
      for (int j = 0; j < 3; ++j) nsum(&s[j], &cc[j], creal(gb * hm[j]));
    }
    for (int j = 0; j < 3; ++j)
      for (int c = 0; c < 3; ++c) corner[9 * m + 3 * j + c] = (s[j] + cc[j]) * N[c];
  }
  /* gather corners to vertices in face order (deterministic) */
  double* acc = (double*)calloc((size_t)(3 * n_verts), sizeof(double));
  if (!acc) { free(corner); free(want); return 1; }
  for (int64_t m = 0; m < n_faces; ++m)
    for (int j = 0; j < 3; ++j)
      for (int c = 0; c < 3; ++c) acc[3 * faces[3 * m + j] + c] += corner[9 * m + 3 * j + c];
  if (vsel) {
    for (int64_t i = 0; i < n_sel; ++i)
      for (int c = 0; c < 3; ++c) grad[3 * i + c] = acc[3 * vsel[i] + c];
  } else {
    memcpy(grad, acc, sizeof(double) * 3 * (size_t)n_verts);
  }
  free(acc); free(corner); free(want);
  return 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
