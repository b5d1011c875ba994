/*
 * Plain FP64 CPU oracle for Levenberg-Marquardt optimisation of a Sim(3)
 * essential graph, the pose-graph step of loop correction in FastLoop
 * (Sec. III-B: pose graph optimisation over the essential graph propagates
 * the loop correction; Sec. IV-F: Graphite LM with automatically
 * differentiated Jacobians and an exact LDL^T linear solve; Sec. VI:
 * a Levenberg-Marquardt scheme).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path and must never be used as a
 * fallback for it.
 *
 * Everything here follows the mathematical definitions directly, with no
 * blocking or fusion beyond what the definitions state:
 *   - exp of the Sim(3) generator is the matrix exponential of the 4x4
 *     generator (Taylor series with scaling and squaring);
 *   - the V matrix W in log is its defining series sum_n X^n/(n+1)!;
 *   - the left Jacobian is sum_n ad^n/(n+1)! and its inverse is obtained by
 *     Gaussian elimination (no closed forms, no Bernoulli series);
 *   - the damped normal equations are solved exactly by a block sparse
 *     Cholesky factorisation with a minimum-degree ordering (the paper uses
 *     an exact LDL^T; both give the same solution up to rounding).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   pose S = (R, t, s) maps world to camera, x -> s R x + t;
 *   tangent order xi = [omega, upsilon, sigma], left perturbation exp(d) S;
 *   edge residual r = log(Z S_i S_j^-1), Z ~ S_j S_i^-1;
 *   cost F = sum_e w_e r_e^T Omega_e r_e (no 1/2);
 *   b = sum w A^T Omega r, H = sum w A^T Omega A, step (H + lambda I) d = -b;
 *   gain ratio rho = (F - F') / (d^T (lambda d - b));
 *   accept if rho > 0: lambda *= max(1/3, 1-(2 rho-1)^3), nu = 2,
 *   else lambda *= nu, nu *= 2;  lambda_0 = tau * max diag(H);
 *   one fixed gauge vertex; quaternions renormalised after each update.
 *
 * Around the optimisation, the loop-correction steps of Sec. III-B: the
 * connected keyframes take the loop's Sim(3) correction before it
 * (og_propagate_correction) and map points follow their reference keyframe
 * (og_correct_points), both written as the compositions they are.
 *
 * Parity pins (tests): exp/log round trips and the closed-form limits of the
 * V matrix, central finite differences of the Jacobians, zero cost on
 * noise-free graphs, gauge invariance of the final cost, the closed-form
 * translation-only ring, dense and scipy cross-checks of the linear solve,
 * and brute-force finite differences of the whole solve for the adjoint;
 * for the loop correction a hand-worked example, the identity correction,
 * the closed form of a change of world frame and the invariance of a point
 * in its reference camera.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------ */
/* small dense linear algebra                                          */
/* ------------------------------------------------------------------ */

/* C(n x m) = A(n x k) * B(k x m), row-major; C must not alias A or B */
static void mm(const double *A, const double *B, double *C, int n, int k, int m) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      double acc = 0.0;
      for (int l = 0; l < k; ++l) acc += A[i * k + l] * B[l * m + j];
      C[i * m + j] = acc;
    }
}

/* C(n x m) = A(k x n)^T * B(k x m) */
static void mtm(const double *A, const double *B, double *C, int n, int k, int m) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      double acc = 0.0;
      for (int l = 0; l < k; ++l) acc += A[l * n + i] * B[l * m + j];
      C[i * m + j] = acc;
    }
}

/* Solve A X = B for X (A n x n, B n x m), Gaussian elimination with partial
 * pivoting; A and B are overwritten, X returned in B.  Returns 0 on success. */
static int gauss_solve(double *A, double *B, int n, int m) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = fabs(A[c * n + c]);
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > best) { best = fabs(A[r * n + c]); p = r; }
    if (!(best > 0.0)) return -1;
    if (p != c) {
      for (int j = 0; j < n; ++j) { double t = A[c * n + j]; A[c * n + j] = A[p * n + j]; A[p * n + j] = t; }
      for (int j = 0; j < m; ++j) { double t = B[c * m + j]; B[c * m + j] = B[p * m + j]; B[p * m + j] = t; }
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      if (f == 0.0) continue;
      for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
      for (int j = 0; j < m; ++j) B[r * m + j] -= f * B[c * m + j];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    for (int j = 0; j < m; ++j) {
      double acc = B[c * m + j];
      for (int l = c + 1; l < n; ++l) acc -= A[c * n + l] * B[l * m + j];
      B[c * m + j] = acc / A[c * n + c];
    }
  }
  return 0;
}

/* In-place lower Cholesky of a 7x7 SPD block (upper part zeroed). */
static int chol7(double *A) {
  for (int j = 0; j < 7; ++j) {
    double d = A[j * 7 + j];
    for (int k = 0; k < j; ++k) d -= A[j * 7 + k] * A[j * 7 + k];
    if (!(d > 0.0) || !isfinite(d)) return -1;
    d = sqrt(d);
    A[j * 7 + j] = d;
    for (int i = j + 1; i < 7; ++i) {
      double s = A[i * 7 + j];
      for (int k = 0; k < j; ++k) s -= A[i * 7 + k] * A[j * 7 + k];
      A[i * 7 + j] = s / d;
    }
    for (int i = 0; i < j; ++i) A[i * 7 + j] = 0.0;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Sim(3)                                                              */
/* ------------------------------------------------------------------ */
typedef struct { double R[9]; double t[3]; double s; } sim3;

static void quat_to_R(const double *q_in, double *R) {
  double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
  double x = q_in[0] / n, y = q_in[1] / n, z = q_in[2] / n, w = q_in[3] / n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Rotation matrix -> unit quaternion (x, y, z, w) with w >= 0 (Shepperd). */
static void R_to_quat(const double *R, double *q) {
  double tr = R[0] + R[4] + R[8];
  double x, y, z, w;
  if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
    double r = sqrt(1.0 + tr) * 2.0;
    w = 0.25 * r; x = (R[7] - R[5]) / r; y = (R[2] - R[6]) / r; z = (R[3] - R[1]) / r;
  } else if (R[0] >= R[4] && R[0] >= R[8]) {
    double r = sqrt(1.0 + R[0] - R[4] - R[8]) * 2.0;
    x = 0.25 * r; y = (R[1] + R[3]) / r; z = (R[2] + R[6]) / r; w = (R[7] - R[5]) / r;
  } else if (R[4] >= R[8]) {
    double r = sqrt(1.0 + R[4] - R[0] - R[8]) * 2.0;
    y = 0.25 * r; x = (R[1] + R[3]) / r; z = (R[5] + R[7]) / r; w = (R[2] - R[6]) / r;
  } else {
    double r = sqrt(1.0 + R[8] - R[0] - R[4]) * 2.0;
    z = 0.25 * r; x = (R[2] + R[6]) / r; y = (R[5] + R[7]) / r; w = (R[3] - R[1]) / r;
  }
  if (w < 0) { x = -x; y = -y; z = -z; w = -w; }
  double n = sqrt(x * x + y * y + z * z + w * w);
  q[0] = x / n; q[1] = y / n; q[2] = z / n; q[3] = w / n;
}

static sim3 sim3_from8(const double *p) {
  sim3 S;
  quat_to_R(p, S.R);
  S.t[0] = p[4]; S.t[1] = p[5]; S.t[2] = p[6]; S.s = p[7];
  return S;
}

static void sim3_to8(const sim3 *S, double *p) {
  R_to_quat(S->R, p);
  p[4] = S->t[0]; p[5] = S->t[1]; p[6] = S->t[2]; p[7] = S->s;
}

/* a * b = (R_a R_b, s_a R_a t_b + t_a, s_a s_b) */
static sim3 sim3_mul(const sim3 *a, const sim3 *b) {
  sim3 c;
  mm(a->R, b->R, c.R, 3, 3, 3);
  double Rt[3];
  mm(a->R, b->t, Rt, 3, 3, 1);
  for (int k = 0; k < 3; ++k) c.t[k] = a->s * Rt[k] + a->t[k];
  c.s = a->s * b->s;
  return c;
}

/* a^-1 = (R^T, -R^T t / s, 1 / s) */
static sim3 sim3_inv(const sim3 *a) {
  sim3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c.R[i * 3 + j] = a->R[j * 3 + i];
  double Rt[3];
  mm(c.R, a->t, Rt, 3, 3, 1);
  for (int k = 0; k < 3; ++k) c.t[k] = -Rt[k] / a->s;
  c.s = 1.0 / a->s;
  return c;
}

static void hat3(const double *w, double *W) {
  W[0] = 0;     W[1] = -w[2]; W[2] = w[1];
  W[3] = w[2];  W[4] = 0;     W[5] = -w[0];
  W[6] = -w[1]; W[7] = w[0];  W[8] = 0;
}

/* Matrix exponential of an n x n matrix (n <= 8): Taylor series of the
 * matrix scaled below norm 1/2, then repeated squaring. */
static void expm(const double *X, double *E, int n) {
  double norm = 0.0;
  for (int i = 0; i < n; ++i) {
    double row = 0.0;
    for (int j = 0; j < n; ++j) row += fabs(X[i * n + j]);
    if (row > norm) norm = row;
  }
  int k = 0;
  while (norm > 0.5) { norm *= 0.5; ++k; }
  double scale = ldexp(1.0, -k);
  double Y[64], term[64], tmp[64];
  for (int i = 0; i < n * n; ++i) Y[i] = X[i] * scale;
  for (int i = 0; i < n * n; ++i) { E[i] = 0.0; term[i] = 0.0; }
  for (int i = 0; i < n; ++i) { E[i * n + i] = 1.0; term[i * n + i] = 1.0; }
  for (int m = 1; m <= 30; ++m) {
    mm(term, Y, tmp, n, n, n);
    double mx = 0.0;
    for (int i = 0; i < n * n; ++i) { term[i] = tmp[i] / m; E[i] += term[i]; if (fabs(term[i]) > mx) mx = fabs(term[i]); }
    if (mx < 1e-20) break;
  }
  for (int s = 0; s < k; ++s) {
    mm(E, E, tmp, n, n, n);
    memcpy(E, tmp, sizeof(double) * n * n);
  }
}

/* exp of the generator xi = [omega, upsilon, sigma]:
 * the 4x4 matrix [[omega^ + sigma I, upsilon], [0, 0]] exponentiated. */
static sim3 sim3_exp(const double *xi) {
  double X[16] = {0};
  double W[9];
  hat3(xi, W);
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) X[i * 4 + j] = W[i * 3 + j] + (i == j ? xi[6] : 0.0);
    X[i * 4 + 3] = xi[3 + i];
  }
  double M[16];
  expm(X, M, 4);
  sim3 S;
  S.s = exp(xi[6]);
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) S.R[i * 3 + j] = M[i * 4 + j] / S.s;
    S.t[i] = M[i * 4 + 3];
  }
  return S;
}

/* W(omega, sigma) = sum_{n>=0} X^n / (n+1)!,  X = omega^ + sigma I */
static void sim3_W(const double *omega, double sigma, double *Wm) {
  double X[9], term[9], tmp[9];
  hat3(omega, X);
  for (int i = 0; i < 3; ++i) X[i * 3 + i] += sigma;
  for (int i = 0; i < 9; ++i) { term[i] = (i % 4 == 0) ? 1.0 : 0.0; Wm[i] = term[i]; }
  for (int n = 1; n < 400; ++n) {
    mm(term, X, tmp, 3, 3, 3);
    double mx = 0.0, wx = 0.0;
    for (int i = 0; i < 9; ++i) {
      term[i] = tmp[i] / (n + 1);
      Wm[i] += term[i];
      if (fabs(term[i]) > mx) mx = fabs(term[i]);
      if (fabs(Wm[i]) > wx) wx = fabs(Wm[i]);
    }
    if (mx <= 1e-19 * wx) break;
  }
}

/* log: sigma = ln s, omega = rotation vector of R, upsilon = W^-1 t. */
static void sim3_log(const sim3 *S, double *xi) {
  double q[4];
  R_to_quat(S->R, q);
  double nv = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
  double f = 0.0;
  if (nv > 0.0) f = 2.0 * atan2(nv, q[3]) / nv;
  double omega[3] = {f * q[0], f * q[1], f * q[2]};
  double sigma = log(S->s);
  double Wm[9], rhs[3] = {S->t[0], S->t[1], S->t[2]};
  sim3_W(omega, sigma, Wm);
  gauss_solve(Wm, rhs, 3, 1);
  xi[0] = omega[0]; xi[1] = omega[1]; xi[2] = omega[2];
  xi[3] = rhs[0]; xi[4] = rhs[1]; xi[5] = rhs[2];
  xi[6] = sigma;
}

/* Adj(S) in [omega, upsilon, sigma] order: [[R,0,0],[t^R, sR, -t],[0,0,1]] */
static void sim3_adj(const sim3 *S, double *A) {
  double th[9], tR[9];
  hat3(S->t, th);
  mm(th, S->R, tR, 3, 3, 3);
  memset(A, 0, sizeof(double) * 49);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      A[i * 7 + j] = S->R[i * 3 + j];
      A[(3 + i) * 7 + j] = tR[i * 3 + j];
      A[(3 + i) * 7 + 3 + j] = S->s * S->R[i * 3 + j];
    }
  for (int i = 0; i < 3; ++i) A[(3 + i) * 7 + 6] = -S->t[i];
  A[48] = 1.0;
}

/* ad(xi) = [[omega^,0,0],[upsilon^, omega^ + sigma I, -upsilon],[0,0,0]] */
static void sim3_ad(const double *xi, double *ad) {
  double wh[9], uh[9];
  hat3(xi, wh);
  hat3(xi + 3, uh);
  memset(ad, 0, sizeof(double) * 49);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      ad[i * 7 + j] = wh[i * 3 + j];
      ad[(3 + i) * 7 + j] = uh[i * 3 + j];
      ad[(3 + i) * 7 + 3 + j] = wh[i * 3 + j] + (i == j ? xi[6] : 0.0);
    }
  for (int i = 0; i < 3; ++i) ad[(3 + i) * 7 + 6] = -xi[3 + i];
}

/* Left Jacobian J_l(xi) = sum_{n>=0} ad(xi)^n / (n+1)!  (exp(xi + dx) =
 * exp(J_l dx) exp(xi) to first order). */
static void left_jacobian(const double *xi, double *J) {
  double ad[49], term[49], tmp[49];
  sim3_ad(xi, ad);
  for (int i = 0; i < 49; ++i) { term[i] = (i % 8 == 0) ? 1.0 : 0.0; J[i] = term[i]; }
  for (int n = 1; n < 400; ++n) {
    mm(term, ad, tmp, 7, 7, 7);
    double mx = 0.0, jx = 0.0;
    for (int i = 0; i < 49; ++i) {
      term[i] = tmp[i] / (n + 1);
      J[i] += term[i];
      if (fabs(term[i]) > mx) mx = fabs(term[i]);
      if (fabs(J[i]) > jx) jx = fabs(J[i]);
    }
    if (mx <= 1e-19 * jx) break;
  }
}

/* ------------------------------------------------------------------ */
/* graph                                                               */
/* ------------------------------------------------------------------ */
typedef struct {
  int K;            /* number of free vertices */
  int *perm;        /* elimination position -> vertex */
  int *pos;         /* vertex -> elimination position (-1 for the fixed vertex) */
  int64_t *colptr;  /* K+1, entries of column k: rows (positions > k), sorted */
  int *rowpos;
  double *L;        /* 49 per entry */
  double *D;        /* 49 per column: the diagonal Cholesky factor */
  int64_t nnz;
} chol_t;

typedef struct {
  int n, m, fixed;
  int *ei, *ej;
  sim3 *Z;
  double *w;
  double *info;     /* NULL = identity */
  chol_t ch;
} ograph;

static void info_mul(const ograph *g, int e, const double *v, double *out, int ncols) {
  /* out(7 x ncols) = Omega_e * v(7 x ncols) */
  if (!g->info) { memcpy(out, v, sizeof(double) * 7 * ncols); return; }
  mm(g->info + (size_t)e * 49, v, out, 7, 7, ncols);
}

/* Residual r = log(Z S_i S_j^-1) and (optionally) exact Jacobians
 * A_i = dr/d(delta_i) = J_l^-1(r) Adj(Z), A_j = -J_l^-1(r) Adj(T),
 * T = Z S_i S_j^-1, for left perturbations exp(delta) S. */
static int edge_eval(const sim3 *Z, const sim3 *Si, const sim3 *Sj,
                     double *r, double *Ai, double *Aj) {
  sim3 Sji = sim3_inv(Sj);
  sim3 P = sim3_mul(Si, &Sji);
  sim3 T = sim3_mul(Z, &P);
  sim3_log(&T, r);
  if (!Ai) return 0;
  double J[49], Jc[49], B[98];
  left_jacobian(r, J);
  double AdZ[49], AdT[49];
  sim3_adj(Z, AdZ);
  sim3_adj(&T, AdT);
  for (int i = 0; i < 7; ++i)
    for (int j = 0; j < 7; ++j) {
      B[i * 14 + j] = AdZ[i * 7 + j];
      B[i * 14 + 7 + j] = -AdT[i * 7 + j];
    }
  memcpy(Jc, J, sizeof(J));
  if (gauss_solve(Jc, B, 7, 14)) return -1;
  for (int i = 0; i < 7; ++i)
    for (int j = 0; j < 7; ++j) {
      Ai[i * 7 + j] = B[i * 14 + j];
      Aj[i * 7 + j] = B[i * 14 + 7 + j];
    }
  return 0;
}

static sim3 *poses_from8(const ograph *g, const double *p) {
  sim3 *S = (sim3 *)malloc(sizeof(sim3) * (size_t)g->n);
  for (int v = 0; v < g->n; ++v) S[v] = sim3_from8(p + (size_t)v * 8);
  return S;
}

/* F = sum_e w_e r_e^T Omega_e r_e */
static double cost_sim3(const ograph *g, const sim3 *S, double *r_out) {
  double F = 0.0;
  for (int e = 0; e < g->m; ++e) {
    double r[7], Or[7];
    edge_eval(&g->Z[e], &S[g->ei[e]], &S[g->ej[e]], r, NULL, NULL);
    info_mul(g, e, r, Or, 1);
    double c = 0.0;
    for (int k = 0; k < 7; ++k) c += r[k] * Or[k];
    F += g->w[e] * c;
    if (r_out) memcpy(r_out + (size_t)e * 7, r, sizeof(r));
  }
  return F;
}

/* ---------------- minimum-degree ordering and symbolic factor -------- */
typedef struct { int *a; int n, cap; } ivec;

static void iv_push(ivec *v, int x) {
  if (v->n == v->cap) { v->cap = v->cap ? 2 * v->cap : 8; v->a = (int *)realloc(v->a, sizeof(int) * v->cap); }
  v->a[v->n++] = x;
}

static int cmp_int(const void *a, const void *b) { int x = *(const int *)a, y = *(const int *)b; return (x > y) - (x < y); }

static void iv_sort_unique(ivec *v) {
  if (v->n == 0) return;
  qsort(v->a, v->n, sizeof(int), cmp_int);
  int k = 1;
  for (int i = 1; i < v->n; ++i) if (v->a[i] != v->a[k - 1]) v->a[k++] = v->a[i];
  v->n = k;
}

/* out = (a U b) \ {x, y}; a, b sorted unique */
static void iv_merge_excl(const ivec *a, const int *b, int nb, int x, int y, ivec *out) {
  out->n = 0;
  int i = 0, j = 0;
  while (i < a->n || j < nb) {
    int v;
    if (j >= nb || (i < a->n && a->a[i] < b[j])) v = a->a[i++];
    else if (i >= a->n || b[j] < a->a[i]) v = b[j++];
    else { v = a->a[i]; ++i; ++j; }
    if (v != x && v != y) iv_push(out, v);
  }
}

static int symbolic(ograph *g) {
  int n = g->n;
  chol_t *c = &g->ch;
  c->K = n - 1;
  ivec *adj = (ivec *)calloc((size_t)n, sizeof(ivec));
  for (int e = 0; e < g->m; ++e) {
    int i = g->ei[e], j = g->ej[e];
    if (i == g->fixed || j == g->fixed) continue;
    iv_push(&adj[i], j);
    iv_push(&adj[j], i);
  }
  for (int v = 0; v < n; ++v) iv_sort_unique(&adj[v]);
  char *done = (char *)calloc((size_t)n, 1);
  done[g->fixed] = 1;
  c->perm = (int *)malloc(sizeof(int) * (size_t)(c->K > 0 ? c->K : 1));
  c->pos = (int *)malloc(sizeof(int) * (size_t)n);
  for (int v = 0; v < n; ++v) c->pos[v] = -1;
  ivec *structv = (ivec *)calloc((size_t)n, sizeof(ivec));
  ivec tmp = {0};
  for (int k = 0; k < c->K; ++k) {
    int best = -1, bd = 0;
    for (int v = 0; v < n; ++v) {
      if (done[v]) continue;
      if (best < 0 || adj[v].n < bd) { best = v; bd = adj[v].n; }
    }
    int v = best;
    c->perm[k] = v;
    c->pos[v] = k;
    done[v] = 1;
    /* column structure of v = its current neighbours */
    structv[v].n = 0;
    for (int q = 0; q < adj[v].n; ++q) iv_push(&structv[v], adj[v].a[q]);
    /* eliminate: neighbours become a clique */
    for (int q = 0; q < adj[v].n; ++q) {
      int u = adj[v].a[q];
      iv_merge_excl(&adj[u], adj[v].a, adj[v].n, u, v, &tmp);
      ivec sw = adj[u]; adj[u] = tmp; tmp = sw;
    }
    adj[v].n = 0;
  }
  /* column pointers over elimination positions */
  c->colptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(c->K + 1));
  c->colptr[0] = 0;
  for (int k = 0; k < c->K; ++k) c->colptr[k + 1] = c->colptr[k] + structv[c->perm[k]].n;
  c->nnz = c->colptr[c->K];
  c->rowpos = (int *)malloc(sizeof(int) * (size_t)(c->nnz > 0 ? c->nnz : 1));
  for (int k = 0; k < c->K; ++k) {
    ivec *s = &structv[c->perm[k]];
    int64_t b = c->colptr[k];
    for (int q = 0; q < s->n; ++q) c->rowpos[b + q] = c->pos[s->a[q]];
    qsort(c->rowpos + b, (size_t)s->n, sizeof(int), cmp_int);
  }
  c->L = (double *)malloc(sizeof(double) * 49 * (size_t)(c->nnz > 0 ? c->nnz : 1));
  c->D = (double *)malloc(sizeof(double) * 49 * (size_t)(c->K > 0 ? c->K : 1));
  for (int v = 0; v < n; ++v) { free(adj[v].a); free(structv[v].a); }
  free(adj); free(structv); free(done); free(tmp.a);
  return 0;
}

static int64_t find_entry(const chol_t *c, int col, int row) {
  int64_t lo = c->colptr[col], hi = c->colptr[col + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    int r = c->rowpos[mid];
    if (r == row) return mid;
    if (r < row) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* Numeric factorisation of (H + lambda I) restricted to the free vertices.
 * Hdiag: N x 49, Hoff: per edge (i, j) block H_ij (49, row-major). */
static int numeric(ograph *g, const double *Hdiag, const double *Hoff, double lambda) {
  chol_t *c = &g->ch;
  memset(c->L, 0, sizeof(double) * 49 * (size_t)(c->nnz > 0 ? c->nnz : 1));
  for (int k = 0; k < c->K; ++k) {
    int v = c->perm[k];
    memcpy(c->D + (size_t)k * 49, Hdiag + (size_t)v * 49, sizeof(double) * 49);
    for (int d = 0; d < 7; ++d) c->D[(size_t)k * 49 + d * 8] += lambda;
  }
  for (int e = 0; e < g->m; ++e) {
    int i = g->ei[e], j = g->ej[e];
    if (i == g->fixed || j == g->fixed) continue;
    int pi = c->pos[i], pj = c->pos[j];
    const double *O = Hoff + (size_t)e * 49;   /* block (i, j) */
    if (pi > pj) {
      int64_t q = find_entry(c, pj, pi);
      if (q < 0) return -2;
      for (int a = 0; a < 49; ++a) c->L[q * 49 + a] += O[a];
    } else {
      int64_t q = find_entry(c, pi, pj);
      if (q < 0) return -2;
      for (int a = 0; a < 7; ++a)
        for (int b = 0; b < 7; ++b) c->L[q * 49 + a * 7 + b] += O[b * 7 + a];
    }
  }
  double tmp[49];
  for (int k = 0; k < c->K; ++k) {
    double *Lkk = c->D + (size_t)k * 49;
    if (chol7(Lkk)) return -1;
    /* L_rk = A_rk L_kk^-T : solve X L_kk^T = A_rk row by row */
    for (int64_t q = c->colptr[k]; q < c->colptr[k + 1]; ++q) {
      double *X = c->L + q * 49;
      for (int row = 0; row < 7; ++row)
        for (int col = 0; col < 7; ++col) {
          double s = X[row * 7 + col];
          for (int l = 0; l < col; ++l) s -= X[row * 7 + l] * Lkk[col * 7 + l];
          X[row * 7 + col] = s / Lkk[col * 7 + col];
        }
    }
    /* Schur complement update of the trailing columns */
    for (int64_t q1 = c->colptr[k]; q1 < c->colptr[k + 1]; ++q1) {
      int r1 = c->rowpos[q1];
      const double *L1 = c->L + q1 * 49;
      for (int64_t q2 = q1; q2 < c->colptr[k + 1]; ++q2) {
        int r2 = c->rowpos[q2];
        const double *L2 = c->L + q2 * 49;
        /* tmp = L2 * L1^T */
        for (int a = 0; a < 7; ++a)
          for (int b = 0; b < 7; ++b) {
            double s = 0.0;
            for (int l = 0; l < 7; ++l) s += L2[a * 7 + l] * L1[b * 7 + l];
            tmp[a * 7 + b] = s;
          }
        double *dst;
        if (r1 == r2) dst = c->D + (size_t)r1 * 49;
        else {
          int64_t q = find_entry(c, r1, r2);
          if (q < 0) return -2;
          dst = c->L + q * 49;
        }
        for (int a = 0; a < 49; ++a) dst[a] -= tmp[a];
      }
    }
  }
  return 0;
}

/* Solve with the current factor: x (N x 7) = (H + lambda I)^-1 rhs on the free
 * vertices, x = 0 on the fixed vertex. */
static void chol_solve(const ograph *g, const double *rhs, double *x) {
  const chol_t *c = &g->ch;
  double *y = (double *)malloc(sizeof(double) * 7 * (size_t)(c->K > 0 ? c->K : 1));
  for (int k = 0; k < c->K; ++k) memcpy(y + (size_t)k * 7, rhs + (size_t)c->perm[k] * 7, sizeof(double) * 7);
  for (int k = 0; k < c->K; ++k) {
    const double *Lkk = c->D + (size_t)k * 49;
    double *yk = y + (size_t)k * 7;
    for (int a = 0; a < 7; ++a) {
      double s = yk[a];
      for (int l = 0; l < a; ++l) s -= Lkk[a * 7 + l] * yk[l];
      yk[a] = s / Lkk[a * 8];
    }
    for (int64_t q = c->colptr[k]; q < c->colptr[k + 1]; ++q) {
      double *yr = y + (size_t)c->rowpos[q] * 7;
      const double *Lq = c->L + q * 49;
      for (int a = 0; a < 7; ++a) {
        double s = 0.0;
        for (int l = 0; l < 7; ++l) s += Lq[a * 7 + l] * yk[l];
        yr[a] -= s;
      }
    }
  }
  for (int k = c->K - 1; k >= 0; --k) {
    double *yk = y + (size_t)k * 7;
    for (int64_t q = c->colptr[k]; q < c->colptr[k + 1]; ++q) {
      const double *yr = y + (size_t)c->rowpos[q] * 7;
      const double *Lq = c->L + q * 49;
      for (int a = 0; a < 7; ++a) {
        double s = 0.0;
        for (int l = 0; l < 7; ++l) s += Lq[l * 7 + a] * yr[l];
        yk[a] -= s;
      }
    }
    const double *Lkk = c->D + (size_t)k * 49;
    for (int a = 6; a >= 0; --a) {
      double s = yk[a];
      for (int l = a + 1; l < 7; ++l) s -= Lkk[l * 7 + a] * yk[l];
      yk[a] = s / Lkk[a * 8];
    }
  }
  memset(x, 0, sizeof(double) * 7 * (size_t)g->n);
  for (int k = 0; k < c->K; ++k) memcpy(x + (size_t)c->perm[k] * 7, y + (size_t)k * 7, sizeof(double) * 7);
  free(y);
}

/* ------------------------------------------------------------------ */
/* exported API                                                        */
/* ------------------------------------------------------------------ */
EXPORT void *og_create(int n, int m, int fixed, const int32_t *ei, const int32_t *ej,
                       const double *meas, const double *w, const double *info) {
  if (n < 1 || m < 0 || fixed < 0 || fixed >= n) return NULL;
  for (int e = 0; e < m; ++e)
    if (ei[e] < 0 || ei[e] >= n || ej[e] < 0 || ej[e] >= n || ei[e] == ej[e]) return NULL;
  ograph *g = (ograph *)calloc(1, sizeof(ograph));
  g->n = n; g->m = m; g->fixed = fixed;
  g->ei = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
  g->ej = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
  g->Z = (sim3 *)malloc(sizeof(sim3) * (size_t)(m > 0 ? m : 1));
  g->w = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  for (int e = 0; e < m; ++e) {
    g->ei[e] = ei[e]; g->ej[e] = ej[e];
    g->Z[e] = sim3_from8(meas + (size_t)e * 8);
    g->w[e] = w ? w[e] : 1.0;
  }
  if (info) {
    g->info = (double *)malloc(sizeof(double) * 49 * (size_t)(m > 0 ? m : 1));
    memcpy(g->info, info, sizeof(double) * 49 * (size_t)m);
  }
  symbolic(g);
  return g;
}

EXPORT void og_destroy(void *h) {
  ograph *g = (ograph *)h;
  if (!g) return;
  free(g->ei); free(g->ej); free(g->Z); free(g->w); free(g->info);
  free(g->ch.perm); free(g->ch.pos); free(g->ch.colptr); free(g->ch.rowpos);
  free(g->ch.L); free(g->ch.D);
  free(g);
}

EXPORT int64_t og_factor_nnz(void *h) { return ((ograph *)h)->ch.nnz; }

EXPORT void og_exp(const double *xi, double *pose8) { sim3 S = sim3_exp(xi); sim3_to8(&S, pose8); }

EXPORT void og_log(const double *pose8, double *xi) { sim3 S = sim3_from8(pose8); sim3_log(&S, xi); }

EXPORT void og_W(const double *omega, double sigma, double *Wm) { sim3_W(omega, sigma, Wm); }

EXPORT void og_left_jacobian(const double *xi, double *J) { left_jacobian(xi, J); }

EXPORT void og_adj(const double *pose8, double *A) { sim3 S = sim3_from8(pose8); sim3_adj(&S, A); }

EXPORT void og_compose(const double *a8, const double *b8, double *c8) {
  sim3 a = sim3_from8(a8), b = sim3_from8(b8);
  sim3 c = sim3_mul(&a, &b);
  sim3_to8(&c, c8);
}

EXPORT void og_inverse(const double *a8, double *c8) {
  sim3 a = sim3_from8(a8);
  sim3 c = sim3_inv(&a);
  sim3_to8(&c, c8);
}

/* cost F and per-edge residuals r (E x 7, nullable) */
EXPORT double og_cost(void *h, const double *poses, double *r_out) {
  ograph *g = (ograph *)h;
  sim3 *S = poses_from8(g, poses);
  double F = cost_sim3(g, S, r_out);
  free(S);
  return F;
}

/* Exact Jacobians per edge: Ai, Aj (E x 49 each, row-major 7x7) */
EXPORT int og_jacobians(void *h, const double *poses, double *Ai, double *Aj) {
  ograph *g = (ograph *)h;
  sim3 *S = poses_from8(g, poses);
  int rc = 0;
  for (int e = 0; e < g->m; ++e) {
    double r[7];
    if (edge_eval(&g->Z[e], &S[g->ei[e]], &S[g->ej[e]], r, Ai + (size_t)e * 49, Aj + (size_t)e * 49)) rc = -1;
  }
  free(S);
  return rc;
}

/* Normal equations: Hdiag (N x 49) = sum w A^T Omega A per endpoint,
 * Hoff (E x 49) = w A_i^T Omega A_j (the (i, j) block of each edge),
 * b (N x 7) = sum w A^T Omega r.  No rows are dropped here; the fixed vertex
 * is removed by the solve.  Returns the cost F. */
static double linearize_sim3(ograph *g, const sim3 *S, double *Hdiag, double *Hoff, double *b) {
  memset(Hdiag, 0, sizeof(double) * 49 * (size_t)g->n);
  memset(b, 0, sizeof(double) * 7 * (size_t)g->n);
  double F = 0.0;
  for (int e = 0; e < g->m; ++e) {
    int i = g->ei[e], j = g->ej[e];
    double r[7], Ai[49], Aj[49], OAi[49], OAj[49], Or[7], blk[49], g7[7];
    edge_eval(&g->Z[e], &S[i], &S[j], r, Ai, Aj);
    double w = g->w[e];
    info_mul(g, e, Ai, OAi, 7);
    info_mul(g, e, Aj, OAj, 7);
    info_mul(g, e, r, Or, 1);
    double c = 0.0;
    for (int k = 0; k < 7; ++k) c += r[k] * Or[k];
    F += w * c;
    mtm(Ai, OAi, blk, 7, 7, 7);
    for (int a = 0; a < 49; ++a) Hdiag[(size_t)i * 49 + a] += w * blk[a];
    mtm(Aj, OAj, blk, 7, 7, 7);
    for (int a = 0; a < 49; ++a) Hdiag[(size_t)j * 49 + a] += w * blk[a];
    mtm(Ai, OAj, blk, 7, 7, 7);
    for (int a = 0; a < 49; ++a) Hoff[(size_t)e * 49 + a] = w * blk[a];
    mtm(Ai, Or, g7, 7, 7, 1);
    for (int a = 0; a < 7; ++a) b[(size_t)i * 7 + a] += w * g7[a];
    mtm(Aj, Or, g7, 7, 7, 1);
    for (int a = 0; a < 7; ++a) b[(size_t)j * 7 + a] += w * g7[a];
  }
  return F;
}

EXPORT double og_linearize(void *h, const double *poses, double *Hdiag, double *Hoff, double *b) {
  ograph *g = (ograph *)h;
  sim3 *S = poses_from8(g, poses);
  double F = linearize_sim3(g, S, Hdiag, Hoff, b);
  free(S);
  return F;
}

/* Exact solve of (H + lambda I) delta = -b on the free vertices (given H, b). */
EXPORT int og_solve_system(void *h, const double *Hdiag, const double *Hoff, const double *b,
                           double lambda, double *delta) {
  ograph *g = (ograph *)h;
  int rc = numeric(g, Hdiag, Hoff, lambda);
  if (rc) return rc;
  double *rhs = (double *)malloc(sizeof(double) * 7 * (size_t)g->n);
  for (size_t k = 0; k < 7 * (size_t)g->n; ++k) rhs[k] = -b[k];
  chol_solve(g, rhs, delta);
  free(rhs);
  return 0;
}

/* S_v <- exp(delta_v) S_v for every vertex except the fixed one; the stored
 * quaternion is renormalised. */
static void apply_update(const ograph *g, const sim3 *S, const double *delta, sim3 *out) {
  for (int v = 0; v < g->n; ++v) {
    if (v == g->fixed) { out[v] = S[v]; continue; }
    sim3 E = sim3_exp(delta + (size_t)v * 7);
    sim3 P = sim3_mul(&E, &S[v]);
    double p8[8];
    sim3_to8(&P, p8);
    out[v] = sim3_from8(p8);
  }
}

EXPORT void og_apply_update(void *h, const double *poses, const double *delta, double *out) {
  ograph *g = (ograph *)h;
  sim3 *S = poses_from8(g, poses);
  sim3 *O = (sim3 *)malloc(sizeof(sim3) * (size_t)g->n);
  apply_update(g, S, delta, O);
  for (int v = 0; v < g->n; ++v) {
    if (v == g->fixed) memcpy(out + (size_t)v * 8, poses + (size_t)v * 8, sizeof(double) * 8);
    else sim3_to8(&O[v], out + (size_t)v * 8);
  }
  free(S); free(O);
}

typedef struct {
  int max_iters;
  double tau;
  double lambda_init;   /* > 0 overrides tau * max diag */
  double ftol, gtol;
  int polish_iters;     /* undamped Newton steps after LM (see og_lm) */
} og_options;

typedef struct {
  double initial_cost, final_cost, final_lambda, grad_inf_norm;
  int iterations, accepted, stop_reason, status;
} og_report;

static double grad_inf(const ograph *g, const double *b) {
  double gmax = 0.0;
  for (int v = 0; v < g->n; ++v) {
    if (v == g->fixed) continue;
    for (int k = 0; k < 7; ++k) if (fabs(b[(size_t)v * 7 + k]) > gmax) gmax = fabs(b[(size_t)v * 7 + k]);
  }
  return gmax;
}

/* Levenberg-Marquardt (rules in the file header).  poses (N x 8) in/out.
 * stop_reason: 0 max iterations, 1 |F - F'| <= ftol F (accepted or rejected step),
 * 2 gradient inf-norm <= gtol, 3 lambda overflow.
 * Near the optimum the cost decrease of a step falls below the rounding of
 * F itself (it is quadratic in the gradient), so cost-based acceptance stalls
 * at a gradient of about sqrt(eps F lambda_min).  Where a stationary point is
 * needed to full precision (implicit differentiation of the optimum), up to
 * polish_iters undamped Gauss-Newton steps follow the LM loop, each kept only
 * while it lowers the gradient inf-norm; they do not count as LM iterations. */
EXPORT int og_lm(void *h, double *poses, const og_options *opt, og_report *rep) {
  ograph *g = (ograph *)h;
  int n = g->n;
  sim3 *S = poses_from8(g, poses);
  sim3 *Sn = (sim3 *)malloc(sizeof(sim3) * (size_t)n);
  double *Hd = (double *)malloc(sizeof(double) * 49 * (size_t)n);
  double *Ho = (double *)malloc(sizeof(double) * 49 * (size_t)(g->m > 0 ? g->m : 1));
  double *b = (double *)malloc(sizeof(double) * 7 * (size_t)n);
  double *d = (double *)malloc(sizeof(double) * 7 * (size_t)n);
  double F = cost_sim3(g, S, NULL);
  double lambda = -1.0, nu = 2.0, gmax = 0.0;
  int need_lin = 1, it = 0, acc = 0, stop = 0, status = 0;
  memset(rep, 0, sizeof(*rep));
  rep->initial_cost = F;
  for (it = 0; it < opt->max_iters;) {
    if (need_lin) {
      linearize_sim3(g, S, Hd, Ho, b);
      gmax = 0.0;
      for (int v = 0; v < n; ++v) {
        if (v == g->fixed) continue;
        for (int k = 0; k < 7; ++k) if (fabs(b[(size_t)v * 7 + k]) > gmax) gmax = fabs(b[(size_t)v * 7 + k]);
      }
      if (gmax <= opt->gtol) { stop = 2; break; }
      need_lin = 0;
    }
    if (lambda < 0) {
      if (opt->lambda_init > 0) lambda = opt->lambda_init;
      else {
        double mx = 0.0;
        for (int v = 0; v < n; ++v) {
          if (v == g->fixed) continue;
          for (int k = 0; k < 7; ++k) if (Hd[(size_t)v * 49 + k * 8] > mx) mx = Hd[(size_t)v * 49 + k * 8];
        }
        lambda = opt->tau * mx;
      }
    }
    int rc = og_solve_system(g, Hd, Ho, b, lambda, d);
    ++it;
    double Fn = INFINITY, pred = 0.0;
    if (rc == 0) {
      apply_update(g, S, d, Sn);
      Fn = cost_sim3(g, Sn, NULL);
      for (int v = 0; v < n; ++v)
        for (int k = 0; k < 7; ++k) {
          double dv = d[(size_t)v * 7 + k];
          pred += dv * (lambda * dv - b[(size_t)v * 7 + k]);
        }
    }
    double rho = (pred > 0.0 && isfinite(Fn)) ? (F - Fn) / pred : -1.0;
    /* |F - F'| <= ftol F, accepted or not: no progress is measurable */
    const int flat = isfinite(Fn) && fabs(F - Fn) <= opt->ftol * F;
    if (rho > 0.0) {
      sim3 *sw = S; S = Sn; Sn = sw;
      double f = 2.0 * rho - 1.0;
      f = 1.0 - f * f * f;
      lambda *= (f > 1.0 / 3.0 ? f : 1.0 / 3.0);
      nu = 2.0;
      need_lin = 1;
      ++acc;
      F = Fn;
      if (flat) { stop = 1; break; }
    } else {
      lambda *= nu;
      nu *= 2.0;
      if (flat) { stop = 1; break; }
      if (!(lambda < 1e32)) { stop = 3; break; }
    }
  }
  for (int k = 0; k < opt->polish_iters; ++k) {
    linearize_sim3(g, S, Hd, Ho, b);
    double g0 = grad_inf(g, b);
    gmax = g0;
    if (g0 <= opt->gtol) break;
    if (og_solve_system(g, Hd, Ho, b, 0.0, d)) break;
    apply_update(g, S, d, Sn);
    linearize_sim3(g, Sn, Hd, Ho, b);
    double g1 = grad_inf(g, b);
    if (!(g1 < g0)) break;
    sim3 *sw = S; S = Sn; Sn = sw;
    F = cost_sim3(g, S, NULL);
    gmax = g1;
  }
  for (int v = 0; v < n; ++v) {
    if (v == g->fixed) continue;
    sim3_to8(&S[v], poses + (size_t)v * 8);
  }
  rep->final_cost = F;
  rep->final_lambda = lambda;
  rep->grad_inf_norm = gmax;
  rep->iterations = it;
  rep->accepted = acc;
  rep->stop_reason = stop;
  rep->status = status;
  free(S); free(Sn); free(Hd); free(Ho); free(b); free(d);
  return status;
}

/* ---------------- implicit adjoint ----------------------------------- */

/* Per-edge gradient g_e = [A_i^T Omega r ; A_j^T Omega r] (14, without the
 * weight) at poses exp(di) S_i, exp(dj) S_j and measurement exp(dz) Z. */
static void edge_grad(const ograph *g, int e, const sim3 *Si, const sim3 *Sj,
                      const double *di, const double *dj, const double *dz, double *g14) {
  sim3 Pi = *Si, Pj = *Sj, Zp = g->Z[e];
  if (di) { sim3 E = sim3_exp(di); Pi = sim3_mul(&E, Si); }
  if (dj) { sim3 E = sim3_exp(dj); Pj = sim3_mul(&E, Sj); }
  if (dz) { sim3 E = sim3_exp(dz); Zp = sim3_mul(&E, &g->Z[e]); }
  double r[7], Ai[49], Aj[49], Or[7];
  edge_eval(&Zp, &Pi, &Pj, r, Ai, Aj);
  info_mul(g, e, r, Or, 1);
  mtm(Ai, Or, g14, 7, 7, 1);
  mtm(Aj, Or, g14 + 7, 7, 7, 1);
}

/* Full Hessian of F/2 at the optimum, assembled from per-edge 14 x 14
 * blocks d g_e / d(delta_i, delta_j) taken by central differences (step h)
 * of the exact per-edge gradient, then symmetrised. */
static void full_hessian(const ograph *g, const sim3 *S, double h, double *Hd, double *Ho) {
  memset(Hd, 0, sizeof(double) * 49 * (size_t)g->n);
  for (int e = 0; e < g->m; ++e) {
    int i = g->ei[e], j = g->ej[e];
    double Hloc[196];          /* Hloc[row * 14 + col] = d g_row / d x_col */
    for (int col = 0; col < 14; ++col) {
      double dp[7] = {0}, gp[14], gm[14];
      dp[col % 7] = h;
      if (col < 7) edge_grad(g, e, &S[i], &S[j], dp, NULL, NULL, gp);
      else edge_grad(g, e, &S[i], &S[j], NULL, dp, NULL, gp);
      dp[col % 7] = -h;
      if (col < 7) edge_grad(g, e, &S[i], &S[j], dp, NULL, NULL, gm);
      else edge_grad(g, e, &S[i], &S[j], NULL, dp, NULL, gm);
      for (int row = 0; row < 14; ++row) Hloc[row * 14 + col] = g->w[e] * (gp[row] - gm[row]) / (2.0 * h);
    }
    for (int a = 0; a < 7; ++a)
      for (int c = 0; c < 7; ++c) {
        Hd[(size_t)i * 49 + a * 7 + c] += Hloc[a * 14 + c];
        Hd[(size_t)j * 49 + a * 7 + c] += Hloc[(7 + a) * 14 + 7 + c];
        /* (i, j) block: symmetrise the two off-diagonal 7x7 parts */
        Ho[(size_t)e * 49 + a * 7 + c] = 0.5 * (Hloc[a * 14 + 7 + c] + Hloc[(7 + c) * 14 + a]);
      }
  }
  for (int v = 0; v < g->n; ++v)
    for (int a = 0; a < 7; ++a)
      for (int c = a + 1; c < 7; ++c) {
        double s = 0.5 * (Hd[(size_t)v * 49 + a * 7 + c] + Hd[(size_t)v * 49 + c * 7 + a]);
        Hd[(size_t)v * 49 + a * 7 + c] = s;
        Hd[(size_t)v * 49 + c * 7 + a] = s;
      }
}

/* Implicit differentiation of the optimum x*(z, w) through b(x*, z, w) = 0:
 * mu = H_full^-1 dL/dx, dL/dtheta = -mu^T db/dtheta.
 * dL_dx: N x 7 (left-tangent gradient; the fixed row is ignored).
 * Outputs: dL_dmeas E x 7 (left-tangent perturbation exp(dz) Z_e),
 *          dL_dw E, mu N x 7 (nullable). h: central-difference step. */
EXPORT int og_adjoint(void *hg, const double *poses, const double *dL_dx, double h,
                      double *dL_dmeas, double *dL_dw, double *mu_out) {
  ograph *g = (ograph *)hg;
  sim3 *S = poses_from8(g, poses);
  double *Hd = (double *)malloc(sizeof(double) * 49 * (size_t)g->n);
  double *Ho = (double *)malloc(sizeof(double) * 49 * (size_t)(g->m > 0 ? g->m : 1));
  double *mu = (double *)malloc(sizeof(double) * 7 * (size_t)g->n);
  double *negrhs = (double *)malloc(sizeof(double) * 7 * (size_t)g->n);
  full_hessian(g, S, h, Hd, Ho);
  for (size_t k = 0; k < 7 * (size_t)g->n; ++k) negrhs[k] = -dL_dx[k];
  /* og_solve_system solves (H) x = -rhs */
  int rc = og_solve_system(g, Hd, Ho, negrhs, 0.0, mu);
  if (rc == 0) {
    for (int e = 0; e < g->m; ++e) {
      int i = g->ei[e], j = g->ej[e];
      const double *mi = mu + (size_t)i * 7, *mj = mu + (size_t)j * 7;
      double g14[14];
      edge_grad(g, e, &S[i], &S[j], NULL, NULL, NULL, g14);
      double s = 0.0;
      for (int k = 0; k < 7; ++k) s += mi[k] * g14[k] + mj[k] * g14[7 + k];
      dL_dw[e] = -s;
      for (int d = 0; d < 7; ++d) {
        double dz[7] = {0}, gp[14], gm[14];
        dz[d] = h;
        edge_grad(g, e, &S[i], &S[j], NULL, NULL, dz, gp);
        dz[d] = -h;
        edge_grad(g, e, &S[i], &S[j], NULL, NULL, dz, gm);
        double acc = 0.0;
        for (int k = 0; k < 7; ++k)
          acc += mi[k] * (gp[k] - gm[k]) + mj[k] * (gp[7 + k] - gm[7 + k]);
        dL_dmeas[(size_t)e * 7 + d] = -g->w[e] * acc / (2.0 * h);
      }
    }
    if (mu_out) memcpy(mu_out, mu, sizeof(double) * 7 * (size_t)g->n);
  }
  free(S); free(Hd); free(Ho); free(mu); free(negrhs);
  return rc;
}

/* Pose-error loss L = 1/2 sum_{v != fixed} |log(S_v G_v^-1)|^2 and its
 * left-tangent gradient dL/d(delta_v) = J_l^-T(l_v) l_v (N x 7). */
EXPORT double og_pose_loss(void *hg, const double *poses, const double *gt, double *grad) {
  ograph *g = (ograph *)hg;
  double L = 0.0;
  for (int v = 0; v < g->n; ++v) {
    double *gv = grad ? grad + (size_t)v * 7 : NULL;
    if (v == g->fixed) { if (gv) memset(gv, 0, sizeof(double) * 7); continue; }
    sim3 S = sim3_from8(poses + (size_t)v * 8), G = sim3_from8(gt + (size_t)v * 8);
    sim3 Gi = sim3_inv(&G);
    sim3 D = sim3_mul(&S, &Gi);
    double l[7];
    sim3_log(&D, l);
    for (int k = 0; k < 7; ++k) L += 0.5 * l[k] * l[k];
    if (gv) {
      double J[49], Jt[49], rhs[7];
      left_jacobian(l, J);
      for (int a = 0; a < 7; ++a)
        for (int c = 0; c < 7; ++c) Jt[a * 7 + c] = J[c * 7 + a];
      memcpy(rhs, l, sizeof(l));
      gauss_solve(Jt, rhs, 7, 1);
      memcpy(gv, rhs, sizeof(rhs));
    }
  }
  return L;
}

/* ------------------------------------------------------------------ */
/* Loop correction around the pose graph optimisation (Sec. III-B,     */
/* "Loop Correction")                                                  */
/* ------------------------------------------------------------------ */

/* x -> s R x + t */
static void sim3_apply(const sim3 *S, const double *x, double *y) {
  double Rx[3];
  mm(S->R, x, Rx, 3, 3, 1);
  for (int k = 0; k < 3; ++k) y[k] = S->s * Rx[k] + S->t[k];
}

/* Before the pose graph optimisation the keyframes connected to the current
 * keyframe c take the loop's Sim(3) correction: with S_c' the corrected pose
 * of c (estimated by the loop detection), every listed keyframe k keeps its
 * pose relative to c,
 *     S_k' = (S_k S_c^-1) S_c',
 * and every keyframe not listed keeps its pose (copied).  out: n x 8. */
EXPORT void og_propagate_correction(int n, const double *poses, int current, const double *corrected8,
                                    int n_conn, const int32_t *conn, double *out) {
  memcpy(out, poses, sizeof(double) * 8 * (size_t)n);
  const sim3 Sc = sim3_from8(poses + 8 * (size_t)current);
  const sim3 Scinv = sim3_inv(&Sc);
  const sim3 Sc_new = sim3_from8(corrected8);
  for (int a = 0; a < n_conn; ++a) {
    const int k = conn[a];
    const sim3 Sk = sim3_from8(poses + 8 * (size_t)k);
    const sim3 rel = sim3_mul(&Sk, &Scinv);          /* S_k S_c^-1: camera c -> camera k */
    const sim3 Sk_new = sim3_mul(&rel, &Sc_new);
    sim3_to8(&Sk_new, out + 8 * (size_t)k);
  }
}

/* Map-point correction: a point keeps its position in the camera frame of
 * its reference keyframe r while that keyframe's pose changes from
 * S_before[r] to S_after[r]:
 *     x' = S_after[r]^-1 (S_before[r] x).
 * Points with r < 0 are copied.  X, out: P x 3 (world coordinates). */
EXPORT void og_correct_points(int n, const double *before, const double *after, int P, const double *X,
                              const int32_t *ref, double *out) {
  (void)n;
  for (int p = 0; p < P; ++p) {
    const int r = ref[p];
    if (r < 0) {
      memcpy(out + 3 * (size_t)p, X + 3 * (size_t)p, sizeof(double) * 3);
      continue;
    }
    const sim3 Sb = sim3_from8(before + 8 * (size_t)r);
    const sim3 Sa = sim3_from8(after + 8 * (size_t)r);
    const sim3 Sa_inv = sim3_inv(&Sa);
    double y[3];
    sim3_apply(&Sb, X + 3 * (size_t)p, y);       /* into the reference camera */
    sim3_apply(&Sa_inv, y, out + 3 * (size_t)p); /* back to the corrected world */
  }
}

/* ------------------------------------------------------------------ */
/* Projection search and loop fusion (Sec. IV-D)                       */
/* ------------------------------------------------------------------ */
/* Both project map points into keyframes and match ORB descriptors:
 *   projection search (PS1 / PS3a-c, Sec. IV-D "Single / Triple
 *   Projection Search"): correspondences between map points and a
 *   keyframe's features, skipping features matched before the search;
 *   loop fusion (Sec. IV-D "Loop Fusion"): for every connected keyframe,
 *   the loop map points that duplicate one of its points (descriptor
 *   similarity and spatial proximity) or that it should observe.
 * The per-pair rule (ORB-SLAM lineage; the paper names the operations
 * only), in single precision like the system the paper builds on:
 *   pose (q, t, s) taken to float, R = R(q / |q|);
 *   p = s R x + t; reject if p_z <= 0;
 *   u = fx p_x / p_z + cx, v = fy p_y / p_z + cy; reject outside
 *   [min_x, max_x) x [min_y, max_y);
 *   O = -(R^T t) / s (camera centre), d = |x - O|; reject unless
 *   min_dist <= d <= max_dist, and if (x - O) . n < cos_min d (n the
 *   point's mean viewing direction);
 *   level = smallest L >= 0 with max_dist <= d scale^L (scale^L by
 *   repeated multiplication), at most n_levels - 1;
 *   radius = th scale^level; candidates: features with |u_f - u| < radius,
 *   |v_f - v| < radius and level - 1 <= octave <= level (search: and not
 *   matched before); best = smallest Hamming distance of the 256-bit
 *   descriptors, ties to the lower feature index; a match if best <= th_low.
 * Every floating-point step is one IEEE single operation in a fixed order
 * (no contraction under -std=c99), so a GPU performing the same operations in
 * the same order takes the same decisions.
 * Conflicts (reading; the paper resolves them on the CPU after the kernel):
 *   search: a feature chosen by several points goes to the one with the
 *   smallest (distance, point index); the others get no match;
 *   fusion: if several loop points choose the same feature of a keyframe
 *   that has no map point there, the smallest (distance, point index) adds
 *   its observation and the others fuse with that point; a feature that has
 *   a map point makes every loop point choosing it fuse with that point. */
typedef struct {
  float fx, fy, cx, cy;
  float min_x, max_x, min_y, max_y;
  float scale_factor;
  float th;           /* search radius at level 0, pixels */
  float cos_min;      /* minimum cosine of the viewing angle */
  int n_levels;
  int th_low;         /* largest accepted Hamming distance */
} og_proj_params;

static int popcount32(uint32_t x) {
  int c = 0;
  while (x) { x &= x - 1u; ++c; }
  return c;
}

static int hamming256(const uint32_t *a, const uint32_t *b) {
  int d = 0;
  for (int k = 0; k < 8; ++k) d += popcount32(a[k] ^ b[k]);
  return d;
}

/* One (keyframe, point) pair: the predicted feature index (-1: none) and the
 * Hamming distance of its best candidate (256 if none).  Features of the
 * keyframe: f in [0, nf). */
static int proj_pair(const og_proj_params *pp, const double *pose8, int nf, const float *fu, const float *fv,
                     const int32_t *foct, const uint32_t *fdesc, const uint8_t *fskip,
                     const float *X, const uint32_t *pdesc, float min_dist, float max_dist, const float *nrm,
                     int *best_dist) {
  const float qx = (float)pose8[0], qy = (float)pose8[1], qz = (float)pose8[2], qw = (float)pose8[3];
  const float t0 = (float)pose8[4], t1 = (float)pose8[5], t2 = (float)pose8[6], s = (float)pose8[7];
  const float n = sqrtf(((qx * qx + qy * qy) + qz * qz) + qw * qw);
  const float x = qx / n, y = qy / n, z = qz / n, w = qw / n;
  float R[9];
  R[0] = 1.0f - 2.0f * (y * y + z * z); R[1] = 2.0f * (x * y - w * z);        R[2] = 2.0f * (x * z + w * y);
  R[3] = 2.0f * (x * y + w * z);        R[4] = 1.0f - 2.0f * (x * x + z * z); R[5] = 2.0f * (y * z - w * x);
  R[6] = 2.0f * (x * z - w * y);        R[7] = 2.0f * (y * z + w * x);        R[8] = 1.0f - 2.0f * (x * x + y * y);
  const float px = s * ((R[0] * X[0] + R[1] * X[1]) + R[2] * X[2]) + t0;
  const float py = s * ((R[3] * X[0] + R[4] * X[1]) + R[5] * X[2]) + t1;
  const float pz = s * ((R[6] * X[0] + R[7] * X[1]) + R[8] * X[2]) + t2;
  *best_dist = 256;
  if (!(pz > 0.0f)) return -1;
  const float u = pp->fx * px / pz + pp->cx;
  const float v = pp->fy * py / pz + pp->cy;
  if (u < pp->min_x || u >= pp->max_x || v < pp->min_y || v >= pp->max_y) return -1;
  const float ox = -((R[0] * t0 + R[3] * t1) + R[6] * t2) / s;
  const float oy = -((R[1] * t0 + R[4] * t1) + R[7] * t2) / s;
  const float oz = -((R[2] * t0 + R[5] * t1) + R[8] * t2) / s;
  const float dx = X[0] - ox, dy = X[1] - oy, dz = X[2] - oz;
  const float dist = sqrtf((dx * dx + dy * dy) + dz * dz);
  if (dist < min_dist || dist > max_dist) return -1;
  if ((dx * nrm[0] + dy * nrm[1]) + dz * nrm[2] < pp->cos_min * dist) return -1;
  int level = 0;
  float sc = 1.0f;
  while (level < pp->n_levels - 1 && max_dist > dist * sc) {
    sc = sc * pp->scale_factor;
    ++level;
  }
  const float r = pp->th * sc;   /* sc = scale^level */
  int best = -1, bd = 256;
  for (int f = 0; f < nf; ++f) {
    if (fskip && fskip[f]) continue;
    if (foct[f] < level - 1 || foct[f] > level) continue;
    if (!(fabsf(fu[f] - u) < r) || !(fabsf(fv[f] - v) < r)) continue;
    const int d = hamming256(fdesc + 8 * (size_t)f, pdesc);
    if (d < bd) { bd = d; best = f; }
  }
  *best_dist = bd;
  return bd <= pp->th_low ? best : -1;
}

/* mode 0: projection search, mode 1: loop fusion.  K keyframes with poses
 * (K x 8, double, taken to float) and features in CSR (feat_ptr[K + 1]; fu,
 * fv float, foct int32, fdesc 8 uint32 per feature; fskip: search, nonzero =
 * matched before (nullable); fmp: fusion, the map point id at each feature
 * or -1).  P points (float): X (P x 3), pdesc (P x 8 uint32), min/max
 * distance, normal (P x 3), pid (fusion: the point's map point id; a
 * keyframe with a feature holding that id already observes the point and is
 * skipped).  Outputs K x P: match (feature index within the keyframe or -1),
 * dist (Hamming distance of the best candidate, 256 if none), fuse (fusion:
 * the map point id the point fuses with, -1 = it adds a new observation;
 * search: may be NULL). */
EXPORT void og_project_match(const og_proj_params *pp, int mode, int K, const double *poses, const int32_t *feat_ptr,
                             const float *fu, const float *fv, const int32_t *foct, const uint32_t *fdesc,
                             const uint8_t *fskip, const int32_t *fmp, int P, const float *X, const uint32_t *pdesc,
                             const float *min_dist, const float *max_dist, const float *nrm, const int32_t *pid,
                             int32_t *match, int32_t *dist, int32_t *fuse) {
  for (int k = 0; k < K; ++k) {
    const int f0 = feat_ptr[k], nf = feat_ptr[k + 1] - feat_ptr[k];
    for (int p = 0; p < P; ++p) {
      const size_t o = (size_t)k * P + p;
      int skip_point = 0;
      if (mode == 1)
        for (int f = 0; f < nf; ++f)
          if (fmp[f0 + f] == pid[p]) { skip_point = 1; break; }
      int bd = 256, m = -1;
      if (!skip_point)
        m = proj_pair(pp, poses + 8 * (size_t)k, nf, fu + f0, fv + f0, foct + f0, fdesc + 8 * (size_t)f0,
                      (mode == 0 && fskip) ? fskip + f0 : NULL, X + 3 * (size_t)p, pdesc + 8 * (size_t)p,
                      min_dist[p], max_dist[p], nrm + 3 * (size_t)p, &bd);
      match[o] = m;
      dist[o] = bd;
      if (fuse) fuse[o] = -1;
    }
    /* conflicts within this keyframe: for every feature, the point with the
     * smallest (distance, point index) among those that chose it */
    int32_t *win = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nf > 0 ? nf : 1));
    for (int f = 0; f < nf; ++f) win[f] = -1;
    for (int p = 0; p < P; ++p) {
      const size_t o = (size_t)k * P + p;
      const int m = match[o];
      if (m < 0) continue;
      const int w = win[m];
      if (w < 0 || dist[o] < dist[(size_t)k * P + w]) win[m] = p;   /* p rises: ties keep the lower index */
    }
    for (int p = 0; p < P; ++p) {
      const size_t o = (size_t)k * P + p;
      const int m = match[o];
      if (m < 0) continue;
      if (mode == 0) {
        if (win[m] != p) { match[o] = -1; dist[o] = 256; }
      } else {
        const int existing = fmp[f0 + m];
        if (existing >= 0) fuse[o] = existing;
        else if (win[m] != p) fuse[o] = pid[win[m]];
      }
    }
    free(win);
  }
}
