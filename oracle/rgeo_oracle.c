/*
 * rgeo_oracle.c -- plain FP64 CPU oracle for the geodesic ray tracer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code,
 * header, table or helper with the CUDA path; both sides only consume the
 * same seeded input arrays.
 *
 * Every function follows the paper ("Design and visualization of Riemannian
 * metrics", Novello, da Silva, Velho 2020) in its own notation, slowly and
 * literally:
 *   - metric coefficients in coordinates, Eq. 3.1;
 *   - geodesic flow, Eq. 3.3, with the Christoffel symbols written out as a
 *     full 3x3x3 tensor and contracted against the velocity;
 *   - graph metric g = I + grad f grad f^T (Eq. 5.2) and its Christoffel
 *     symbols Gamma^m_ij = f_m f_ij / (1 + |grad f|^2) (Eq. 5.3);
 *   - pull-back metric g = J^T J (Eq. 5.6) and Theorem 5.1,
 *     Gamma^m_ij = sum_s d_i d_j x_s [J^-1]_ms, with J^-1 from the signed
 *     minors (the unnumbered formula before Theorem 5.1);
 *   - Gaussian bump of Eq. 6.1, summed as in Section 6 ("Summing functions");
 *   - the twist map of Section 5.2;
 *   - Euler marching (Eq. 4.1), or classical RK4 (mentioned in Section 4.1),
 *     with every polygon segment tested against the scene (Section 4.1);
 *   - Riemannian shading: one ray per direction of the view field (Section 4).
 *
 * Readings of the paper used here (also listed in the design notes):
 *   - Eq. 3.4 is read as Gamma^m_ij = 1/2 sum_k g^mk (d_i g_jk + d_j g_ik - d_k g_ij);
 *   - the initial tangent is g-unit (a point of the unit sphere S^2_p of T_pM);
 *   - each bump is truncated at ||(x - c)/sigma|| < cutoff.  Outside every
 *     truncated support, with no quadratic part, Hess f = 0 and the ray is a
 *     straight line, so it is advanced in closed form to the next support
 *     ball (exact for the truncated metric);
 *   - segment parameter s in [0, s_max); a segment starting inside a sphere
 *     hits it at s = 0; triangles are two-sided and edge-inclusive;
 *     ties go to the smaller s, then spheres before triangles, then lower id;
 *     the triangle test is the watertight one of Woop, Benthin and Wald (2013);
 *   - Lambert headlight shading albedo * (0.1 + 0.9 max(0, -n.v)), or
 *     pseudo-colour rgb = clamp(0.5 + hit / 8), rgba8 = floor(255 c + 0.5).
 *
 * Random numbers: none.  Threads: pixels are split over POSIX threads with a
 * static interleave; each pixel's computation is independent and sequential.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_GRAPH 0
#define OR_TWIST 1
#define OR_LOCAL 2
#define OR_RK4 0
#define OR_EULER 1
#define OR_LAMBERT 0
#define OR_PSEUDO 1

#define OR_MISS (-1)
#define OR_BUDGET (-2)

/* ------------------------------------------------------------------ metric */

typedef struct {
  int kind;        /* OR_GRAPH, OR_TWIST or OR_LOCAL */
  int K;           /* number of Gaussian bumps (OR_LOCAL: of composed local maps) */
  double *c;       /* [K*3] centres (x0, y0, z0) of Eq. 6.1 */
  double *a;       /* [K] amplitudes a */
  double *sig;     /* [K*3] spreads sigma_x, sigma_y, sigma_z */
  double b[3];     /* affine part of f: b . x */
  double A[9];     /* quadratic part of f: 1/2 x^T A x (A symmetric, row-major) */
  double cutoff;   /* truncation radius in units of sigma; <= 0 means none */
  double k;        /* twist rate: Phi rotates by k z about the z axis */
  double *dir;     /* OR_LOCAL: [K*3] directions v_i of Phi_i(p) = p + f_i(p) V_i(p) */
  double *Bf;      /* OR_LOCAL: [K*9] field matrices, V_i(p) = v_i + B_i (p - c_i) */
} or_metric;

or_metric *or_metric_create(int kind, int K, const double *c, const double *a,
                            const double *sig, const double *b, const double *A,
                            double cutoff, double k) {
  or_metric *m = (or_metric *)calloc(1, sizeof(or_metric));
  m->kind = kind;
  m->K = K;
  m->c = (double *)malloc(sizeof(double) * 3 * (K > 0 ? K : 1));
  m->a = (double *)malloc(sizeof(double) * (K > 0 ? K : 1));
  m->sig = (double *)malloc(sizeof(double) * 3 * (K > 0 ? K : 1));
  if (K > 0) {
    memcpy(m->c, c, sizeof(double) * 3 * K);
    memcpy(m->a, a, sizeof(double) * K);
    memcpy(m->sig, sig, sizeof(double) * 3 * K);
  }
  for (int i = 0; i < 3; i++) m->b[i] = b ? b[i] : 0.0;
  for (int i = 0; i < 9; i++) m->A[i] = A ? A[i] : 0.0;
  m->cutoff = cutoff;
  m->k = k;
  return m;
}

/* Directions and field matrices of an OR_LOCAL metric (B may be NULL: constant V_i = v_i). */
void or_metric_set_local(or_metric *m, const double *dir, const double *B) {
  int K = m->K > 0 ? m->K : 1;
  m->dir = (double *)calloc(3 * (size_t)K, sizeof(double));
  m->Bf = (double *)calloc(9 * (size_t)K, sizeof(double));
  if (m->K > 0) {
    memcpy(m->dir, dir, sizeof(double) * 3 * m->K);
    if (B) memcpy(m->Bf, B, sizeof(double) * 9 * m->K);
  }
}

void or_metric_destroy(or_metric *m) {
  if (!m) return;
  free(m->dir);
  free(m->Bf);
  free(m->c);
  free(m->a);
  free(m->sig);
  free(m);
}

/* f, its gradient and its Hessian at x for the graph function
 * f = b.x + 1/2 x^T A x + sum_k f_k, with f_k the Gaussian of Eq. 6.1
 * (Section 6, "Summing functions": derivatives of a sum are sums).
 * d f_k / d x_i     = -f_k (x_i - x0_i) / sigma_i^2
 * d2 f_k / dx_i dx_j = f_k [ (x_i - x0_i)(x_j - x0_j) / (sigma_i^2 sigma_j^2) - delta_ij / sigma_i^2 ] */
void or_field(const or_metric *m, const double x[3], double *f_out, double grad[3],
              double hess[9]) {
  double f = 0.0;
  for (int i = 0; i < 3; i++) {
    f += m->b[i] * x[i];
    grad[i] = m->b[i];
    for (int j = 0; j < 3; j++) {
      f += 0.5 * x[i] * m->A[3 * i + j] * x[j];
      grad[i] += m->A[3 * i + j] * x[j];
      hess[3 * i + j] = m->A[3 * i + j];
    }
  }
  for (int k = 0; k < m->K; k++) {
    double d[3], s2[3], u = 0.0;
    for (int i = 0; i < 3; i++) {
      d[i] = x[i] - m->c[3 * k + i];
      s2[i] = m->sig[3 * k + i] * m->sig[3 * k + i];
      u += d[i] * d[i] / s2[i];
    }
    if (m->cutoff > 0.0 && u >= m->cutoff * m->cutoff) continue;
    double fk = m->a[k] * exp(-0.5 * u);
    f += fk;
    for (int i = 0; i < 3; i++) {
      grad[i] += -fk * d[i] / s2[i];
      for (int j = 0; j < 3; j++) {
        double dij = (i == j) ? 1.0 / s2[i] : 0.0;
        hess[3 * i + j] += fk * (d[i] * d[j] / (s2[i] * s2[j]) - dij);
      }
    }
  }
  if (f_out) *f_out = f;
}

/* Twist map of Section 5.2, Phi(x,y,z) = (cos(kz) x - sin(kz) y, sin(kz) x + cos(kz) y, z). */
void or_twist_phi(double k, const double p[3], double out[3]) {
  double c = cos(k * p[2]), s = sin(k * p[2]);
  out[0] = c * p[0] - s * p[1];
  out[1] = s * p[0] + c * p[1];
  out[2] = p[2];
}

/* Inverse of the twist: rotate (X, Y) back by -k Z. */
void or_twist_phi_inv(double k, const double q[3], double out[3]) {
  double c = cos(k * q[2]), s = sin(k * q[2]);
  out[0] = c * q[0] + s * q[1];
  out[1] = -s * q[0] + c * q[1];
  out[2] = q[2];
}

/* Jacobian J[s][i] = d x_s / d x_i of the twist (row s = component of Phi). */
void or_twist_jacobian(double k, const double p[3], double J[9]) {
  double c = cos(k * p[2]), s = sin(k * p[2]);
  double x = p[0], y = p[1];
  J[0] = c;  J[1] = -s; J[2] = -k * (s * x + c * y);
  J[3] = s;  J[4] = c;  J[5] = k * (c * x - s * y);
  J[6] = 0;  J[7] = 0;  J[8] = 1;
}

/* Hessians H[s][i][j] = d2 x_s / dx_i dx_j of the twist components. */
void or_twist_hessian(double k, const double p[3], double H[27]) {
  double c = cos(k * p[2]), s = sin(k * p[2]);
  double x = p[0], y = p[1];
  memset(H, 0, sizeof(double) * 27);
  /* x_1 = c x - s y */
  H[0 * 9 + 0 * 3 + 2] = H[0 * 9 + 2 * 3 + 0] = -k * s;
  H[0 * 9 + 1 * 3 + 2] = H[0 * 9 + 2 * 3 + 1] = -k * c;
  H[0 * 9 + 2 * 3 + 2] = -k * k * (c * x - s * y);
  /* x_2 = s x + c y */
  H[1 * 9 + 0 * 3 + 2] = H[1 * 9 + 2 * 3 + 0] = k * c;
  H[1 * 9 + 1 * 3 + 2] = H[1 * 9 + 2 * 3 + 1] = -k * s;
  H[1 * 9 + 2 * 3 + 2] = -k * k * (s * x + c * y);
  /* x_3 = z: all second derivatives vanish */
}

static double det3(const double M[9]) {
  return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
         M[2] * (M[3] * M[7] - M[4] * M[6]);
}

/* [J^-1]_ms = (-1)^(s+m) det J_sm / det J, J_sm = J without row s and column m
 * (the unnumbered minors formula preceding Theorem 5.1). */
void or_inverse_by_minors(const double J[9], double Jinv[9]) {
  double dJ = det3(J);
  for (int m = 0; m < 3; m++)
    for (int s = 0; s < 3; s++) {
      double minor[4];
      int n = 0;
      for (int r = 0; r < 3; r++) {
        if (r == s) continue;
        for (int col = 0; col < 3; col++) {
          if (col == m) continue;
          minor[n++] = J[3 * r + col];
        }
      }
      double dm = minor[0] * minor[3] - minor[1] * minor[2];
      double sign = ((s + m) % 2 == 0) ? 1.0 : -1.0;
      Jinv[3 * m + s] = sign * dm / dJ;
    }
}

/* ------------------------------------------------- local diffeomorphisms */

/* One local map Phi_i(p) = p + f_i(p) V_i(p) (the local diffeomorphism of Section 6,
 * "Using diffeomorphism"), with f_i the Gaussian of Eq. 6.1 (isotropic spread sigma_i,
 * not truncated) and the vector field V_i(p) = v_i + B_i (p - c_i).
 * out = Phi_i(p); J[s*3+j] = d_j (Phi_i)_s; H[s*9+i*3+j] = d_i d_j (Phi_i)_s:
 *   d_j (Phi_i)_s = delta_sj + f_j V_s + f B_sj,
 *   d_i d_j (Phi_i)_s = f_ij V_s + f_j B_si + f_i B_sj   (V is affine). */
void or_local_map(const or_metric *m, int idx, const double p[3], double out[3], double J[9], double H[27]) {
  const double *c = m->c + 3 * idx, *v = m->dir + 3 * idx, *B = m->Bf + 9 * idx;
  double sg = m->sig[3 * idx], q = 1.0 / (sg * sg);
  double d[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
  double f = m->a[idx] * exp(-0.5 * q * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
  double gr[3], hs[9], V[3];
  for (int i = 0; i < 3; i++) gr[i] = -q * d[i] * f;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) hs[3 * i + j] = f * (q * q * d[i] * d[j] - (i == j ? q : 0.0));
  for (int s = 0; s < 3; s++) V[s] = v[s] + B[3 * s] * d[0] + B[3 * s + 1] * d[1] + B[3 * s + 2] * d[2];
  for (int s = 0; s < 3; s++) {
    out[s] = p[s] + f * V[s];
    for (int j = 0; j < 3; j++) J[3 * s + j] = (s == j ? 1.0 : 0.0) + gr[j] * V[s] + f * B[3 * s + j];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++)
        H[9 * s + 3 * i + j] = hs[3 * i + j] * V[s] + gr[j] * B[3 * s + i] + gr[i] * B[3 * s + j];
  }
}

/* The composition Phi = Phi_1 o Phi_2 o ... o Phi_K (Section 6, "Composing diffeomorphisms";
 * array index K-1 is applied first).  Built from the inside out with Psi_K = Phi_K and
 * Psi_j = Phi_j o Psi_{j+1}:
 *   J(Psi_j)_p = J(Phi_j)_{Psi_{j+1}(p)} J(Psi_{j+1})_p                       (chain rule)
 *   H(x_s o Psi_{j+1})_p = J(Psi_{j+1})^T_p H(x_s)_{Psi_{j+1}(p)} J(Psi_{j+1})_p
 *                          + sum_r d_r x_s(Psi_{j+1}(p)) H((Psi_{j+1})_r)_p          (Eq. 6.3)
 * with x_s the s-th coordinate of Phi_j.  out = Phi(p). */
void or_local_compose(const or_metric *m, const double p[3], double out[3], double J[9], double H[27]) {
  double q[3], Jj[9], Hj[27], q2[3], Jn[9], Hn[27];
  or_local_map(m, m->K - 1, p, q, J, H);
  for (int j = m->K - 2; j >= 0; j--) {
    or_local_map(m, j, q, q2, Jj, Hj);
    for (int s = 0; s < 3; s++)
      for (int c = 0; c < 3; c++) {
        double acc = 0.0;
        for (int r = 0; r < 3; r++) acc += Jj[3 * s + r] * J[3 * r + c];
        Jn[3 * s + c] = acc;
      }
    for (int s = 0; s < 3; s++)
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
          double acc = 0.0;
          for (int k = 0; k < 3; k++)
            for (int l = 0; l < 3; l++) acc += J[3 * k + a] * Hj[9 * s + 3 * k + l] * J[3 * l + b];
          for (int r = 0; r < 3; r++) acc += Jj[3 * s + r] * H[9 * r + 3 * a + b];
          Hn[9 * s + 3 * a + b] = acc;
        }
    memcpy(q, q2, sizeof(q));
    memcpy(J, Jn, sizeof(Jn));
    memcpy(H, Hn, sizeof(Hn));
  }
  memcpy(out, q, sizeof(q));
}

/* J^-1 of the composition as the paper writes it: J^-1(Phi) = J^-1(Phi_K) ... J^-1(Phi_1),
 * each factor inverted by the signed minors at its own point Psi_{j+1}(p). */
void or_local_jinv(const or_metric *m, const double p[3], double Jinv[9]) {
  double q[3], Ji[9], Hi[27], inv[9], q2[3], acc[9];
  /* points: Phi_K acts at p, Phi_j at Psi_{j+1}(p) */
  double *pts = (double *)malloc(sizeof(double) * 3 * (size_t)m->K);
  memcpy(q, p, sizeof(q));
  for (int j = m->K - 1; j >= 0; j--) {
    memcpy(pts + 3 * j, q, sizeof(q));
    or_local_map(m, j, q, q2, Ji, Hi);
    memcpy(q, q2, sizeof(q));
  }
  /* product J^-1(Phi_K) ... J^-1(Phi_1): start from the right, J^-1(Phi_1) */
  for (int i = 0; i < 9; i++) Jinv[i] = (i % 4 == 0) ? 1.0 : 0.0;
  for (int j = 0; j < m->K; j++) {
    or_local_map(m, j, pts + 3 * j, q2, Ji, Hi);
    or_inverse_by_minors(Ji, inv);
    for (int r = 0; r < 3; r++)
      for (int c = 0; c < 3; c++) {
        double t = 0.0;
        for (int k = 0; k < 3; k++) t += inv[3 * r + k] * Jinv[3 * k + c];
        acc[3 * r + c] = t;
      }
    memcpy(Jinv, acc, sizeof(acc));
  }
  free(pts);
}

/* Metric coefficients g_ij at x: Eq. 5.2 (graph) or Eq. 5.6 (pull-back). */
void or_metric_tensor(const or_metric *m, const double x[3], double g[9]) {
  if (m->kind == OR_GRAPH) {
    double f, gr[3], H[9];
    or_field(m, x, &f, gr, H);
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) g[3 * i + j] = (i == j ? 1.0 : 0.0) + gr[i] * gr[j];
  } else {
    double J[9];
    if (m->kind == OR_LOCAL) {
      double q[3], H[27];
      or_local_compose(m, x, q, J, H);
    } else {
      or_twist_jacobian(m->k, x, J);
    }
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) {
        double s = 0.0;
        for (int kk = 0; kk < 3; kk++) s += J[3 * kk + i] * J[3 * kk + j];
        g[3 * i + j] = s;
      }
  }
}

/* <u, v>_p = sum_ij u_i v_j g_ij(p), Eq. 3.1. */
double or_inner(const or_metric *m, const double p[3], const double u[3], const double v[3]) {
  double g[9], s = 0.0;
  or_metric_tensor(m, p, g);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) s += u[i] * v[j] * g[3 * i + j];
  return s;
}

/* Christoffel symbols Gam[m][i][j] (index m*9 + i*3 + j). */
void or_christoffel(const or_metric *m, const double x[3], double Gam[27]) {
  if (m->kind == OR_GRAPH) {
    /* Eq. 5.3 */
    double f, gr[3], H[9];
    or_field(m, x, &f, gr, H);
    double den = 1.0 + gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
    for (int mm = 0; mm < 3; mm++)
      for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) Gam[mm * 9 + i * 3 + j] = gr[mm] * H[3 * i + j] / den;
  } else {
    /* Theorem 5.1 (Eq. 5.7) */
    double J[9], Jinv[9], H[27];
    if (m->kind == OR_LOCAL) {
      double q[3];
      or_local_compose(m, x, q, J, H);
      or_local_jinv(m, x, Jinv);
    } else {
      or_twist_jacobian(m->k, x, J);
      or_inverse_by_minors(J, Jinv);
      or_twist_hessian(m->k, x, H);
    }
    for (int mm = 0; mm < 3; mm++)
      for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
          double s = 0.0;
          for (int ss = 0; ss < 3; ss++) s += H[ss * 9 + i * 3 + j] * Jinv[3 * mm + ss];
          Gam[mm * 9 + i * 3 + j] = s;
        }
  }
}

/* Geodesic flow right-hand side, Eq. 3.3: y'_k = -sum_ij Gamma^k_ij y_i y_j. */
void or_accel(const or_metric *m, const double x[3], const double v[3], double acc[3]) {
  double Gam[27];
  or_christoffel(m, x, Gam);
  for (int kk = 0; kk < 3; kk++) {
    double s = 0.0;
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) s += Gam[kk * 9 + i * 3 + j] * v[i] * v[j];
    acc[kk] = -s;
  }
}

/* One step of length h on the flow (x' = v, v' = acc(x, v)).
 * Euler: Eq. 4.1.  RK4: classical Runge-Kutta on the same first-order system. */
void or_step(const or_metric *m, int integrator, double h, double x[3], double v[3]) {
  if (integrator == OR_EULER) {
    double a[3];
    or_accel(m, x, v, a);
    for (int i = 0; i < 3; i++) {
      x[i] = x[i] + h * v[i];
      v[i] = v[i] + h * a[i];
    }
    return;
  }
  double x1[3], v1[3], a1[3], x2[3], v2[3], a2[3], x3[3], v3[3], a3[3], x4[3], v4[3], a4[3];
  for (int i = 0; i < 3; i++) { x1[i] = x[i]; v1[i] = v[i]; }
  or_accel(m, x1, v1, a1);
  for (int i = 0; i < 3; i++) { x2[i] = x[i] + 0.5 * h * v1[i]; v2[i] = v[i] + 0.5 * h * a1[i]; }
  or_accel(m, x2, v2, a2);
  for (int i = 0; i < 3; i++) { x3[i] = x[i] + 0.5 * h * v2[i]; v3[i] = v[i] + 0.5 * h * a2[i]; }
  or_accel(m, x3, v3, a3);
  for (int i = 0; i < 3; i++) { x4[i] = x[i] + h * v3[i]; v4[i] = v[i] + h * a3[i]; }
  or_accel(m, x4, v4, a4);
  for (int i = 0; i < 3; i++) {
    x[i] = x[i] + h / 6.0 * (v1[i] + 2.0 * v2[i] + 2.0 * v3[i] + v4[i]);
    v[i] = v[i] + h / 6.0 * (a1[i] + 2.0 * a2[i] + 2.0 * a3[i] + a4[i]);
  }
}

/* n fixed steps from (p, v); writes the polygon p_0..p_n and velocities. */
void or_integrate(const or_metric *m, int integrator, double h, int n, const double p[3],
                  const double v[3], double *xs, double *vs) {
  double x[3] = {p[0], p[1], p[2]}, w[3] = {v[0], v[1], v[2]};
  for (int i = 0; i < 3; i++) { xs[i] = x[i]; vs[i] = w[i]; }
  for (int s = 1; s <= n; s++) {
    or_step(m, integrator, h, x, w);
    for (int i = 0; i < 3; i++) { xs[3 * s + i] = x[i]; vs[3 * s + i] = w[i]; }
  }
}

/* Adaptive Dormand-Prince 5(4) reference (Dormand and Prince 1980), used to
 * measure the discretisation error of the fixed-step integrators.  Integrates
 * the flow from (p, v) over arc parameter T; returns the number of accepted
 * steps, or -1 if the step size collapsed. */
int or_dopri5(const or_metric *m, const double p[3], const double v[3], double T, double rtol,
              double atol, double xT[3], double vT[3]) {
  static const double c2 = 1.0 / 5, c3 = 3.0 / 10, c4 = 4.0 / 5, c5 = 8.0 / 9;
  static const double a21 = 1.0 / 5;
  static const double a31 = 3.0 / 40, a32 = 9.0 / 40;
  static const double a41 = 44.0 / 45, a42 = -56.0 / 15, a43 = 32.0 / 9;
  static const double a51 = 19372.0 / 6561, a52 = -25360.0 / 2187, a53 = 64448.0 / 6561,
                      a54 = -212.0 / 729;
  static const double a61 = 9017.0 / 3168, a62 = -355.0 / 33, a63 = 46732.0 / 5247,
                      a64 = 49.0 / 176, a65 = -5103.0 / 18656;
  static const double b1 = 35.0 / 384, b3 = 500.0 / 1113, b4 = 125.0 / 192, b5 = -2187.0 / 6784,
                      b6 = 11.0 / 84;
  static const double e1 = 35.0 / 384 - 5179.0 / 57600, e3 = 500.0 / 1113 - 7571.0 / 16695,
                      e4 = 125.0 / 192 - 393.0 / 640, e5 = -2187.0 / 6784 + 92097.0 / 339200,
                      e6 = 11.0 / 84 - 187.0 / 2100, e7 = -1.0 / 40;
  (void)c2; (void)c3; (void)c4; (void)c5;
  double y[6] = {p[0], p[1], p[2], v[0], v[1], v[2]};
  double t = 0.0, h = 1e-3;
  int accepted = 0;
  double k[7][6], yt[6], yn[6];
#define OR_F(dst, src)                       \
  do {                                       \
    double xx[3] = {src[0], src[1], src[2]}; \
    double vv[3] = {src[3], src[4], src[5]}; \
    double aa[3];                            \
    or_accel(m, xx, vv, aa);                 \
    dst[0] = vv[0]; dst[1] = vv[1]; dst[2] = vv[2]; \
    dst[3] = aa[0]; dst[4] = aa[1]; dst[5] = aa[2]; \
  } while (0)
  OR_F(k[0], y);
  while (t < T) {
    if (t + h > T) h = T - t;
    for (int i = 0; i < 6; i++) yt[i] = y[i] + h * a21 * k[0][i];
    OR_F(k[1], yt);
    for (int i = 0; i < 6; i++) yt[i] = y[i] + h * (a31 * k[0][i] + a32 * k[1][i]);
    OR_F(k[2], yt);
    for (int i = 0; i < 6; i++) yt[i] = y[i] + h * (a41 * k[0][i] + a42 * k[1][i] + a43 * k[2][i]);
    OR_F(k[3], yt);
    for (int i = 0; i < 6; i++)
      yt[i] = y[i] + h * (a51 * k[0][i] + a52 * k[1][i] + a53 * k[2][i] + a54 * k[3][i]);
    OR_F(k[4], yt);
    for (int i = 0; i < 6; i++)
      yt[i] = y[i] + h * (a61 * k[0][i] + a62 * k[1][i] + a63 * k[2][i] + a64 * k[3][i] +
                          a65 * k[4][i]);
    OR_F(k[5], yt);
    for (int i = 0; i < 6; i++)
      yn[i] = y[i] + h * (b1 * k[0][i] + b3 * k[2][i] + b4 * k[3][i] + b5 * k[4][i] + b6 * k[5][i]);
    OR_F(k[6], yn);
    double err = 0.0;
    for (int i = 0; i < 6; i++) {
      double e = h * (e1 * k[0][i] + e3 * k[2][i] + e4 * k[3][i] + e5 * k[4][i] + e6 * k[5][i] +
                      e7 * k[6][i]);
      double sc = atol + rtol * fmax(fabs(y[i]), fabs(yn[i]));
      err += (e / sc) * (e / sc);
    }
    err = sqrt(err / 6.0);
    if (err <= 1.0) {
      t += h;
      for (int i = 0; i < 6; i++) { y[i] = yn[i]; k[0][i] = k[6][i]; }
      accepted++;
    }
    double fac = (err > 0.0) ? 0.9 * pow(err, -0.2) : 5.0;
    if (fac > 5.0) fac = 5.0;
    if (fac < 0.2) fac = 0.2;
    h *= fac;
    if (h < 1e-14) return -1;
  }
#undef OR_F
  for (int i = 0; i < 3; i++) { xT[i] = y[i]; vT[i] = y[3 + i]; }
  return accepted;
}

/* ------------------------------------------------------------------- scene */

typedef struct {
  double lo[3], hi[3];
  int left, right;  /* children, -1 for a leaf */
  int first, count; /* triangle range in the permuted order (leaves) */
} or_node;

typedef struct {
  int S;
  double *sph;   /* [S*4] centre, radius */
  int T;
  double *tri;   /* [T*9] three vertices per triangle (original order) */
  double *alb;   /* [(S+1)*3] albedo: spheres, then mesh */
  int *perm;     /* triangle ids in BVH order */
  or_node *nodes;
  int n_nodes;
  int use_bvh;
  double fog;       /* fog density per unit of arc length (0: none) */
  double fog_rgb[3];
} or_scene;

static void tri_bounds(const or_scene *sc, int t, double lo[3], double hi[3]) {
  for (int i = 0; i < 3; i++) {
    lo[i] = hi[i] = sc->tri[9 * t + i];
    for (int v = 1; v < 3; v++) {
      double c = sc->tri[9 * t + 3 * v + i];
      if (c < lo[i]) lo[i] = c;
      if (c > hi[i]) hi[i] = c;
    }
  }
}

static double tri_centroid(const or_scene *sc, int t, int axis) {
  return (sc->tri[9 * t + axis] + sc->tri[9 * t + 3 + axis] + sc->tri[9 * t + 6 + axis]) / 3.0;
}

static int g_sort_axis;
static const or_scene *g_sort_scene;
static int cmp_centroid(const void *pa, const void *pb) {
  double ca = tri_centroid(g_sort_scene, *(const int *)pa, g_sort_axis);
  double cb = tri_centroid(g_sort_scene, *(const int *)pb, g_sort_axis);
  if (ca < cb) return -1;
  if (ca > cb) return 1;
  return (*(const int *)pa) - (*(const int *)pb);
}

/* Median split on the longest axis of the node's bounds; leaves hold <= 4 triangles. */
static int bvh_build(or_scene *sc, int first, int count) {
  int id = sc->n_nodes++;
  or_node *nd = &sc->nodes[id];
  for (int i = 0; i < 3; i++) { nd->lo[i] = INFINITY; nd->hi[i] = -INFINITY; }
  for (int q = first; q < first + count; q++) {
    double lo[3], hi[3];
    tri_bounds(sc, sc->perm[q], lo, hi);
    for (int i = 0; i < 3; i++) {
      if (lo[i] < nd->lo[i]) nd->lo[i] = lo[i];
      if (hi[i] > nd->hi[i]) nd->hi[i] = hi[i];
    }
  }
  nd->first = first;
  nd->count = count;
  nd->left = nd->right = -1;
  if (count <= 4) return id;
  int axis = 0;
  double ext = nd->hi[0] - nd->lo[0];
  for (int i = 1; i < 3; i++)
    if (nd->hi[i] - nd->lo[i] > ext) { ext = nd->hi[i] - nd->lo[i]; axis = i; }
  g_sort_axis = axis;
  g_sort_scene = sc;
  qsort(sc->perm + first, count, sizeof(int), cmp_centroid);
  int half = count / 2;
  int l = bvh_build(sc, first, half);
  int r = bvh_build(sc, first + half, count - half);
  sc->nodes[id].left = l;
  sc->nodes[id].right = r;
  sc->nodes[id].count = 0;
  return id;
}

or_scene *or_scene_create(int S, const double *sph, int T, const double *tri, const double *alb,
                          int use_bvh) {
  or_scene *sc = (or_scene *)calloc(1, sizeof(or_scene));
  sc->S = S;
  sc->T = T;
  sc->sph = (double *)malloc(sizeof(double) * 4 * (S > 0 ? S : 1));
  sc->tri = (double *)malloc(sizeof(double) * 9 * (T > 0 ? T : 1));
  sc->alb = (double *)malloc(sizeof(double) * 3 * (S + 1));
  if (S > 0) memcpy(sc->sph, sph, sizeof(double) * 4 * S);
  if (T > 0) memcpy(sc->tri, tri, sizeof(double) * 9 * T);
  memcpy(sc->alb, alb, sizeof(double) * 3 * (S + 1));
  sc->perm = (int *)malloc(sizeof(int) * (T > 0 ? T : 1));
  for (int t = 0; t < T; t++) sc->perm[t] = t;
  sc->nodes = (or_node *)malloc(sizeof(or_node) * (2 * (T > 0 ? T : 1)));
  sc->n_nodes = 0;
  sc->use_bvh = use_bvh && T > 0;
  if (sc->use_bvh) bvh_build(sc, 0, T);
  return sc;
}

/* The fog of the paper's grid figures: a hit's colour c becomes c T + fog_rgb (1 - T) with
 * T = exp(-density * arc length travelled to the hit). */
void or_scene_set_fog(or_scene *sc, double density, const double rgb[3]) {
  sc->fog = density;
  for (int i = 0; i < 3; i++) sc->fog_rgb[i] = rgb ? rgb[i] : 0.0;
}

void or_scene_destroy(or_scene *sc) {
  if (!sc) return;
  free(sc->sph);
  free(sc->tri);
  free(sc->alb);
  free(sc->perm);
  free(sc->nodes);
  free(sc);
}

/* Segment O + s D, s in [0, smax), against a sphere.  Returns 1 and s on a hit.
 * A segment that starts inside or on the sphere hits it at s = 0. */
int or_hit_sphere(const double O[3], const double D[3], double smax, const double sp[4],
                  double *s_out) {
  double oc[3] = {O[0] - sp[0], O[1] - sp[1], O[2] - sp[2]};
  double a = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
  double bh = oc[0] * D[0] + oc[1] * D[1] + oc[2] * D[2];
  double cc = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - sp[3] * sp[3];
  double s;
  if (cc <= 0.0) {
    s = 0.0;
  } else {
    double disc = bh * bh - a * cc;
    if (disc < 0.0 || a <= 0.0) return 0;
    s = (-bh - sqrt(disc)) / a;
    if (s < 0.0) return 0; /* both roots behind the origin */
  }
  if (!(s < smax)) return 0;
  *s_out = s;
  return 1;
}

/* Segment against triangle (v0, v1, v2) with the watertight test of Woop,
 * Benthin and Wald (JCGT 2013): shear the vertices into a frame whose z axis is
 * the segment direction, take the three 2D edge functions there (a shared edge
 * gives exactly opposite values for its two triangles, so no ray leaks between
 * them) and accept when they do not have mixed signs.  Edges are included. */
int or_hit_triangle(const double O[3], const double D[3], double smax, const double *t9,
                    double *s_out) {
  int kz = 0;
  if (fabs(D[1]) > fabs(D[kz])) kz = 1;
  if (fabs(D[2]) > fabs(D[kz])) kz = 2;
  int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
  if (D[kz] < 0.0) { int t = kx; kx = ky; ky = t; }
  if (D[kz] == 0.0) return 0;
  double Sx = D[kx] / D[kz], Sy = D[ky] / D[kz], Sz = 1.0 / D[kz];
  double A[3], B[3], C[3];
  for (int i = 0; i < 3; i++) {
    A[i] = t9[i] - O[i];
    B[i] = t9[3 + i] - O[i];
    C[i] = t9[6 + i] - O[i];
  }
  double Ax = A[kx] - Sx * A[kz], Ay = A[ky] - Sy * A[kz];
  double Bx = B[kx] - Sx * B[kz], By = B[ky] - Sy * B[kz];
  double Cx = C[kx] - Sx * C[kz], Cy = C[ky] - Sy * C[kz];
  double U = Cx * By - Cy * Bx;
  double V = Ax * Cy - Ay * Cx;
  double W = Bx * Ay - By * Ax;
  if ((U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0)) return 0;
  double det = U + V + W;
  if (det == 0.0) return 0;
  double T = U * (Sz * A[kz]) + V * (Sz * B[kz]) + W * (Sz * C[kz]);
  double s = T / det;
  if (!(s >= 0.0 && s < smax)) return 0;
  *s_out = s;
  return 1;
}

static int box_hit(const double lo[3], const double hi[3], const double O[3], const double D[3],
                   double smax) {
  /* slab test on the closed box, slightly inflated so rounding never drops a triangle */
  double t0 = 0.0, t1 = smax;
  for (int i = 0; i < 3; i++) {
    double pad = 1e-9 * (1.0 + fabs(lo[i]) + fabs(hi[i]));
    double l = lo[i] - pad, h = hi[i] + pad;
    if (D[i] == 0.0) {
      if (O[i] < l || O[i] > h) return 0;
      continue;
    }
    double ta = (l - O[i]) / D[i], tb = (h - O[i]) / D[i];
    if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
    if (ta > t0) t0 = ta;
    if (tb < t1) t1 = tb;
    if (t0 > t1) return 0;
  }
  return 1;
}

/* Earliest hit of the segment O + s D, s in [0, smax), against the scene.
 * id in [0, S) for spheres, S + t for triangle t.  Ties: smaller s, then
 * lower id (so spheres before triangles). */
int or_scene_hit(const or_scene *sc, const double O[3], const double D[3], double smax,
                 double *s_out, int *id_out) {
  double best = smax;
  int bid = -1;
  for (int k = 0; k < sc->S; k++) {
    double s;
    if (or_hit_sphere(O, D, smax, sc->sph + 4 * k, &s)) {
      if (bid < 0 || s < best || (s == best && k < bid)) { best = s; bid = k; }
    }
  }
  if (sc->T > 0) {
    if (!sc->use_bvh) {
      for (int t = 0; t < sc->T; t++) {
        double s;
        if (or_hit_triangle(O, D, smax, sc->tri + 9 * t, &s)) {
          int id = sc->S + t;
          if (bid < 0 || s < best || (s == best && id < bid)) { best = s; bid = id; }
        }
      }
    } else {
      int stack[128];
      int sp = 0;
      stack[sp++] = 0;
      while (sp > 0) {
        const or_node *nd = &sc->nodes[stack[--sp]];
        double lim = (bid < 0) ? smax : best;
        /* nodes are visited up to s == best too, so equal-s ties are found */
        if (!box_hit(nd->lo, nd->hi, O, D, lim * (1.0 + 1e-12) + 1e-300)) continue;
        if (nd->left < 0) {
          for (int q = nd->first; q < nd->first + nd->count; q++) {
            int t = sc->perm[q];
            double s;
            if (or_hit_triangle(O, D, smax, sc->tri + 9 * t, &s)) {
              int id = sc->S + t;
              if (bid < 0 || s < best || (s == best && id < bid)) { best = s; bid = id; }
            }
          }
        } else {
          stack[sp++] = nd->left;
          stack[sp++] = nd->right;
        }
      }
    }
  }
  if (bid < 0) return 0;
  *s_out = best;
  *id_out = bid;
  return 1;
}

/* ------------------------------------------------------------------ camera */

typedef struct {
  double pos[3], fwd[3], up[3];
  double vfov_deg;
} or_camera;

static void normalize3(double v[3]) {
  double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  v[0] /= n; v[1] /= n; v[2] /= n;
}

static void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Euclidean unit direction of pixel (i, j): pixel centres, row 0 at the top,
 * vertical field of view, right = up x forward. */
void or_camera_dir(const or_camera *cam, int W, int H, int i, int j, double d[3]) {
  double f[3] = {cam->fwd[0], cam->fwd[1], cam->fwd[2]};
  normalize3(f);
  double r[3];
  cross3(cam->up, f, r);
  normalize3(r);
  double u[3];
  cross3(f, r, u);
  double th = tan(0.5 * cam->vfov_deg * M_PI / 180.0);
  double px = (2.0 * (i + 0.5) / W - 1.0) * th * ((double)W / (double)H);
  double py = (1.0 - 2.0 * (j + 0.5) / H) * th;
  for (int q = 0; q < 3; q++) d[q] = f[q] + px * r[q] + py * u[q];
  normalize3(d);
}

/* --------------------------------------------------------------- the trace */

/* Whether the ray may be advanced in closed form outside the bump supports:
 * graph metric, truncated bumps and no quadratic part (Hess f = 0 there, so
 * by Eq. 5.4 the acceleration vanishes and the geodesic is a straight line). */
static int skippable(const or_metric *m) {
  if (m->kind != OR_GRAPH || !(m->cutoff > 0.0)) return 0;
  for (int i = 0; i < 9; i++)
    if (m->A[i] != 0.0) return 0;
  return 1;
}

static double ball_radius2(const or_metric *m, int k) {
  double s = m->sig[3 * k];
  if (m->sig[3 * k + 1] > s) s = m->sig[3 * k + 1];
  if (m->sig[3 * k + 2] > s) s = m->sig[3 * k + 2];
  return (m->cutoff * s) * (m->cutoff * s);
}

/* x lies outside every ball |x - c_k| < cutoff * max_i sigma_ki (zero-amplitude bumps ignored). */
static int outside_supports(const or_metric *m, const double x[3]) {
  for (int k = 0; k < m->K; k++) {
    if (m->a[k] == 0.0) continue;
    double d0 = x[0] - m->c[3 * k], d1 = x[1] - m->c[3 * k + 1], d2 = x[2] - m->c[3 * k + 2];
    if (d0 * d0 + d1 * d1 + d2 * d2 < ball_radius2(m, k)) return 0;
  }
  return 1;
}

/* Smallest t >= 0 at which x + t v enters a support ball; INFINITY if none. */
static double support_entry(const or_metric *m, const double x[3], const double v[3]) {
  double best = INFINITY;
  double A = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  for (int k = 0; k < m->K; k++) {
    if (m->a[k] == 0.0) continue;
    double o[3] = {x[0] - m->c[3 * k], x[1] - m->c[3 * k + 1], x[2] - m->c[3 * k + 2]};
    double B = o[0] * v[0] + o[1] * v[1] + o[2] * v[2];
    double C = o[0] * o[0] + o[1] * o[1] + o[2] * o[2] - ball_radius2(m, k);
    if (B >= 0.0) continue; /* moving away from (or tangent to) this ball */
    double disc = B * B - A * C;
    if (disc < 0.0) continue;
    double t = (-B - sqrt(disc)) / A;
    if (t < 0.0) t = 0.0;
    if (t < best) best = t;
  }
  return best;
}

typedef struct {
  int32_t *id;
  double *hit;    /* [n*3] */
  int32_t *steps;
  uint8_t *rgba;  /* [n*4] */
  double *drift;
  double *xend;   /* [n*3] final position (diagnostic) */
} or_outputs;

static void shade(const or_scene *sc, int shading, int id, const double P[3], const double D[3], double arc,
                  uint8_t rgba[4]) {
  double rgb[3];
  if (shading == OR_PSEUDO) {
    for (int q = 0; q < 3; q++) rgb[q] = 0.5 + P[q] / 8.0;
  } else {
    double n[3];
    int obj = id < sc->S ? id : sc->S;
    if (id < sc->S) {
      const double *sp = sc->sph + 4 * id;
      for (int q = 0; q < 3; q++) n[q] = P[q] - sp[q];
    } else {
      const double *t9 = sc->tri + 9 * (id - sc->S);
      double e1[3] = {t9[3] - t9[0], t9[4] - t9[1], t9[5] - t9[2]};
      double e2[3] = {t9[6] - t9[0], t9[7] - t9[1], t9[8] - t9[2]};
      cross3(e1, e2, n);
      if (n[0] * D[0] + n[1] * D[1] + n[2] * D[2] > 0.0) {
        n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2];
      }
    }
    normalize3(n);
    double dv[3] = {D[0], D[1], D[2]};
    normalize3(dv);
    double c = -(n[0] * dv[0] + n[1] * dv[1] + n[2] * dv[2]);
    if (c < 0.0) c = 0.0;
    double inten = 0.1 + 0.9 * c;
    for (int q = 0; q < 3; q++) rgb[q] = sc->alb[3 * obj + q] * inten;
  }
  if (sc->fog > 0.0) {
    double T = exp(-sc->fog * arc);
    for (int q = 0; q < 3; q++) rgb[q] = rgb[q] * T + sc->fog_rgb[q] * (1.0 - T);
  }
  for (int q = 0; q < 3; q++) {
    double c = rgb[q] < 0.0 ? 0.0 : (rgb[q] > 1.0 ? 1.0 : rgb[q]);
    rgba[q] = (uint8_t)floor(255.0 * c + 0.5);
  }
  rgba[3] = 255;
}

/* A point light and the parameters of the shooting solve (Riemannian illumination, below). */
typedef struct or_light_s {
  double L[3];
  double h;
  int max_steps;
  int iters;
  double tol;
  double delta;
} or_light;

typedef struct {
  const or_metric *m;
  const or_scene *sc;
  const struct or_light_s *light; /* non-NULL: Riemannian illumination of the hits */
  int32_t *lit;                   /* with light: 1 when lit */
  or_camera cam;
  int W, H;
  double h;
  int max_steps, integrator, shading;
  const int64_t *pixels;
  const double *dirs; /* [n*3] Euclidean initial directions in place of the camera's (or NULL) */
  int64_t n;
  or_outputs out;
  int no_skip; /* pins only: march through flat space step by step */
  int tid, nthreads;
} or_job;

/* One pixel: Riemannian shading of one direction of the view field. */
int or_illuminate_hit(const or_metric *m, const or_scene *sc, const struct or_light_s *lt, int integrator, int id,
                      const double P[3], const double Dhit[3], uint8_t rgba[4], double *cos_out,
                      int *iters_out, double u_out[3]);

static void trace_pixel(const or_job *jb, int64_t q) {
  const or_metric *m = jb->m;
  double d[3];
  if (jb->dirs) {
    for (int c = 0; c < 3; c++) d[c] = jb->dirs[3 * q + c];
    normalize3(d);
  } else {
    int64_t px = jb->pixels[q];
    int i = (int)(px % jb->W), j = (int)(px / jb->W);
    or_camera_dir(&jb->cam, jb->W, jb->H, i, j, d);
  }
  double x[3] = {jb->cam.pos[0], jb->cam.pos[1], jb->cam.pos[2]};
  /* g-unit initial tangent: v = d / sqrt(<d, d>_p) (Eq. 3.1) */
  double nd = sqrt(or_inner(m, x, d, d));
  double v[3] = {d[0] / nd, d[1] / nd, d[2] / nd};
  double e0 = or_inner(m, x, v, v);
  int can_skip = skippable(m) && !jb->no_skip;
  int steps = 0, id = OR_BUDGET;
  /* arc length travelled (for the fog): h per step, s h on the hit chord, and the parameter
   * length of each straight advance (its g-length: the tangent is g-unit) */
  double arc = 0.0;
  double P[3] = {x[0], x[1], x[2]}, Dhit[3] = {v[0], v[1], v[2]};
  for (;;) {
    if (can_skip && outside_supports(m, x)) {
      double t = support_entry(m, x, v);
      double s;
      int hid;
      if (or_scene_hit(jb->sc, x, v, t, &s, &hid)) {
        id = hid;
        for (int c = 0; c < 3; c++) { P[c] = x[c] + s * v[c]; Dhit[c] = v[c]; }
        arc += s;
        break;
      }
      if (isinf(t)) { id = OR_MISS; break; }
      for (int c = 0; c < 3; c++) x[c] = x[c] + t * v[c];
      arc += t;
    }
    if (steps >= jb->max_steps) { id = OR_BUDGET; break; }
    double x0[3] = {x[0], x[1], x[2]};
    or_step(m, jb->integrator, jb->h, x, v);
    steps++;
    double D[3] = {x[0] - x0[0], x[1] - x0[1], x[2] - x0[2]};
    double s;
    int hid;
    if (or_scene_hit(jb->sc, x0, D, 1.0, &s, &hid)) {
      id = hid;
      for (int c = 0; c < 3; c++) { P[c] = x0[c] + s * D[c]; Dhit[c] = D[c]; }
      arc += s * jb->h;
      break;
    }
    arc += jb->h;
  }
  const or_outputs *o = &jb->out;
  o->id[q] = id;
  o->steps[q] = steps;
  if (id >= 0) {
    for (int c = 0; c < 3; c++) o->hit[3 * q + c] = P[c];
    shade(jb->sc, jb->shading, id, P, Dhit, arc, o->rgba + 4 * q);
    if (jb->light)
      jb->lit[q] = or_illuminate_hit(m, jb->sc, jb->light, jb->integrator, id, P, Dhit, o->rgba + 4 * q, NULL,
                                     NULL, NULL);
  } else {
    if (jb->light) jb->lit[q] = 0;
    for (int c = 0; c < 3; c++) o->hit[3 * q + c] = x[c];
    memset(o->rgba + 4 * q, 0, 4);
  }
  if (o->drift) o->drift[q] = or_inner(m, x, v, v) / e0 - 1.0;
  if (o->xend)
    for (int c = 0; c < 3; c++) o->xend[3 * q + c] = x[c];
}

static void *trace_worker(void *arg) {
  or_job *jb = (or_job *)arg;
  for (int64_t q = jb->tid; q < jb->n; q += jb->nthreads) trace_pixel(jb, q);
  return NULL;
}

static int trace_job(const or_metric *m, const or_scene *sc, const struct or_light_s *light, int32_t *lit,
                     const double cam_pos[3], const double cam_fwd[3], const double cam_up[3], double vfov_deg,
                     int W, int H, double h, int max_steps, int integrator, int shading, const int64_t *pixels,
                     int64_t n, int32_t *id, double *hit, int32_t *steps, uint8_t *rgba, double *drift,
                     double *xend, int flags, int nthreads, const double *dirs);

/* Trace the listed pixels (p = j * W + i).  Returns 0 on success. */
int or_trace(const or_metric *m, const or_scene *sc, const double cam_pos[3],
             const double cam_fwd[3], const double cam_up[3], double vfov_deg, int W, int H,
             double h, int max_steps, int integrator, int shading, const int64_t *pixels,
             int64_t n, int32_t *id, double *hit, int32_t *steps, uint8_t *rgba, double *drift,
             double *xend, int flags, int nthreads) {
  return trace_job(m, sc, NULL, NULL, cam_pos, cam_fwd, cam_up, vfov_deg, W, H, h, max_steps, integrator, shading,
                   pixels, n, id, hit, steps, rgba, drift, xend, flags, nthreads, NULL);
}

/* As or_trace for n rays with the given Euclidean initial directions dirs[n*3] (each
 * normalised here) from the camera position, in place of the pixels' directions: the
 * same marching, intersection and shading.  Used to measure how a ray's hit depends on
 * its initial direction. */
int or_trace_dirs(const or_metric *m, const or_scene *sc, const double cam_pos[3], const double *dirs, int64_t n,
                  double h, int max_steps, int integrator, int shading, int32_t *id, double *hit, int32_t *steps,
                  uint8_t *rgba, int nthreads) {
  const double fwd[3] = {0.0, 0.0, 1.0}, up[3] = {0.0, 1.0, 0.0};
  return trace_job(m, sc, NULL, NULL, cam_pos, fwd, up, 60.0, 1, 1, h, max_steps, integrator, shading, NULL, n, id,
                   hit, steps, rgba, NULL, NULL, 0, nthreads, dirs);
}

/* As or_trace, with every hit shaded by Riemannian illumination from the point light
 * (position L; light geodesics with step lh, at most lsteps steps each; at most
 * iters Gauss-Newton steps to a miss of at most tol; difference step delta).
 * lit[q] = 1 when pixel q is lit. */
int or_trace_lit(const or_metric *m, const or_scene *sc, const double cam_pos[3], const double cam_fwd[3],
                 const double cam_up[3], double vfov_deg, int W, int H, double h, int max_steps, int integrator,
                 const double L[3], double lh, int lsteps, int iters, double tol, double delta,
                 const int64_t *pixels, int64_t n, int32_t *id, double *hit, int32_t *steps, uint8_t *rgba,
                 int32_t *lit, int nthreads) {
  or_light lt;
  for (int c = 0; c < 3; c++) lt.L[c] = L[c];
  lt.h = lh;
  lt.max_steps = lsteps;
  lt.iters = iters;
  lt.tol = tol;
  lt.delta = delta;
  return trace_job(m, sc, &lt, lit, cam_pos, cam_fwd, cam_up, vfov_deg, W, H, h, max_steps, integrator, OR_LAMBERT,
                   pixels, n, id, hit, steps, rgba, NULL, NULL, 0, nthreads, NULL);
}

/* Single-hit form for the pins: illumination of hit point P (segment direction D) of object id. */
int or_illuminate(const or_metric *m, const or_scene *sc, const double L[3], double lh, int lsteps, int iters,
                  double tol, double delta, int integrator, int id, const double P[3], const double D[3],
                  uint8_t rgba[4], double *cos_out, int *iters_out, double u_out[3]) {
  or_light lt;
  for (int c = 0; c < 3; c++) lt.L[c] = L[c];
  lt.h = lh;
  lt.max_steps = lsteps;
  lt.iters = iters;
  lt.tol = tol;
  lt.delta = delta;
  return or_illuminate_hit(m, sc, &lt, integrator, id, P, D, rgba, cos_out, iters_out, u_out);
}

static int trace_job(const or_metric *m, const or_scene *sc, const struct or_light_s *light, int32_t *lit,
                     const double cam_pos[3], const double cam_fwd[3], const double cam_up[3], double vfov_deg,
                     int W, int H, double h, int max_steps, int integrator, int shading, const int64_t *pixels,
                     int64_t n, int32_t *id, double *hit, int32_t *steps, uint8_t *rgba, double *drift,
                     double *xend, int flags, int nthreads, const double *dirs) {
  if (nthreads < 1) nthreads = 1;
  or_job base;
  memset(&base, 0, sizeof(base));
  base.m = m;
  base.sc = sc;
  base.light = light;
  base.lit = lit;
  for (int c = 0; c < 3; c++) {
    base.cam.pos[c] = cam_pos[c];
    base.cam.fwd[c] = cam_fwd[c];
    base.cam.up[c] = cam_up[c];
  }
  base.cam.vfov_deg = vfov_deg;
  base.W = W;
  base.H = H;
  base.h = h;
  base.max_steps = max_steps;
  base.integrator = integrator;
  base.shading = shading;
  base.pixels = pixels;
  base.dirs = dirs;
  base.n = n;
  base.out.id = id;
  base.out.hit = hit;
  base.out.steps = steps;
  base.out.rgba = rgba;
  base.out.drift = drift;
  base.out.xend = xend;
  base.nthreads = nthreads;
  base.no_skip = flags & 1;
  or_job *jobs = (or_job *)malloc(sizeof(or_job) * nthreads);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
  for (int t = 0; t < nthreads; t++) {
    jobs[t] = base;
    jobs[t].tid = t;
    if (t > 0) pthread_create(&th[t], NULL, trace_worker, &jobs[t]);
  }
  trace_worker(&jobs[0]);
  for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
  free(jobs);
  free(th);
  return 0;
}

/* ---------------------------------------------------- Riemannian illumination */

/* Section 4 ("Riemannian illumination"): a surface point q is lit by a light
 * source through the geodesics that connect q to it; the radiant intensity is
 * Lambertian and depends on the metric.  Readings (also in the design notes):
 *   - one point light L, direct geodesics only (no indirect ones);
 *   - the geodesic from q to L is found by shooting: a Gauss-Newton solve on the
 *     initial direction d(alpha, beta) = normalize(d0 + alpha e1 + beta e2), with
 *     d0 = normalize(L - q), for a zero miss vector (closest approach of the
 *     marched polygon to L, minus L); the Jacobian by forward differences;
 *   - q = P + 1e-3 n, just off the hit surface along the normal n facing the
 *     incoming ray (as in the headlight shading);
 *   - the Lambert factor is the Riemannian cosine between the surface normal and
 *     the initial tangent u (g-unit): <N, u>_q / |N|_q with N = g^-1 n, that is
 *     n.u / sqrt(n^T g^-1 n); a point is lit when the solve converged, the cosine
 *     is positive and no polygon segment between q and the closest approach to L
 *     meets the scene;
 *   - colour albedo * (0.1 + 0.9 cos) when lit, albedo * 0.1 when not. */


/* Marches the geodesic from q with Euclidean initial direction d until its
 * closest approach to L.  Returns 1 with the miss vector e = closest point - L,
 * or 0 when the step budget ran out first.  With shadow != 0, also tests every
 * polygon segment (and every straight advance) up to the closest point against
 * the scene and sets *blocked. */
static int shoot(const or_metric *m, const or_scene *sc, const or_light *lt, int integrator,
                 const double q[3], const double d[3], double e[3], double u[3], int shadow, int *blocked) {
  double x[3] = {q[0], q[1], q[2]};
  /* g-unit initial tangent along d (Eq. 3.1) */
  const double nd = sqrt(or_inner(m, x, d, d));
  double v[3];
  for (int c = 0; c < 3; c++) u[c] = v[c] = d[c] / nd;
  const int can_skip = skippable(m);
  if (blocked) *blocked = 0;
  int steps = 0;
  for (;;) {
    if (can_skip && outside_supports(m, x)) {
      /* straight line x + t v: closest approach to L at tL, next support ball at te */
      double te = support_entry(m, x, v);
      double w[3] = {lt->L[0] - x[0], lt->L[1] - x[1], lt->L[2] - x[2]};
      double tL = (w[0] * v[0] + w[1] * v[1] + w[2] * v[2]) / (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      if (tL < 0.0) tL = 0.0;
      double tend = tL <= te ? tL : te;
      if (shadow && tend > 0.0) {
        double s;
        int hid;
        if (or_scene_hit(sc, x, v, tend, &s, &hid)) {
          *blocked = 1;
          return 1;
        }
      }
      if (tL <= te) {
        for (int c = 0; c < 3; c++) e[c] = x[c] + tL * v[c] - lt->L[c];
        return 1;
      }
      for (int c = 0; c < 3; c++) x[c] = x[c] + te * v[c];
    }
    if (steps >= lt->max_steps) return 0;
    double x0[3] = {x[0], x[1], x[2]};
    or_step(m, integrator, lt->h, x, v);
    steps++;
    double D[3] = {x[0] - x0[0], x[1] - x0[1], x[2] - x0[2]};
    double w[3] = {lt->L[0] - x0[0], lt->L[1] - x0[1], lt->L[2] - x0[2]};
    double t = (w[0] * D[0] + w[1] * D[1] + w[2] * D[2]) / (D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
    if (t < 1.0) { /* the closest approach lies on this segment (or the distance grows) */
      if (t < 0.0) t = 0.0;
      if (shadow && t > 0.0) {
        double s;
        int hid;
        if (or_scene_hit(sc, x0, D, t, &s, &hid)) {
          *blocked = 1;
          return 1;
        }
      }
      for (int c = 0; c < 3; c++) e[c] = x0[c] + t * D[c] - lt->L[c];
      return 1;
    }
    if (shadow) {
      double s;
      int hid;
      if (or_scene_hit(sc, x0, D, 1.0, &s, &hid)) {
        *blocked = 1;
        return 1;
      }
    }
  }
}

/* Illumination of one hit: P the hit point, Dhit the direction of the segment
 * that hit object id.  Writes the colour and returns 1 when lit (cos_out: the
 * Riemannian cosine, iters_out: Gauss-Newton steps taken, u_out: the initial
 * g-unit tangent). */
int or_illuminate_hit(const or_metric *m, const or_scene *sc, const or_light *lt, int integrator, int id,
                      const double P[3], const double Dhit[3], uint8_t rgba[4], double *cos_out,
                      int *iters_out, double u_out[3]) {
  double n[3];
  int obj = id < sc->S ? id : sc->S;
  if (id < sc->S) {
    const double *sp = sc->sph + 4 * id;
    for (int c = 0; c < 3; c++) n[c] = P[c] - sp[c];
  } else {
    const double *t9 = sc->tri + 9 * (id - sc->S);
    double e1[3] = {t9[3] - t9[0], t9[4] - t9[1], t9[5] - t9[2]};
    double e2[3] = {t9[6] - t9[0], t9[7] - t9[1], t9[8] - t9[2]};
    cross3(e1, e2, n);
  }
  if (n[0] * Dhit[0] + n[1] * Dhit[1] + n[2] * Dhit[2] > 0.0) {
    n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2];
  }
  normalize3(n);
  double q[3];
  for (int c = 0; c < 3; c++) q[c] = P[c] + 1e-3 * n[c];
  double d0[3] = {lt->L[0] - q[0], lt->L[1] - q[1], lt->L[2] - q[2]};
  normalize3(d0);
  /* e1 across the axis least aligned with d0 (lowest index on ties), e2 = d0 x e1 */
  int ax = 0;
  for (int c = 1; c < 3; c++)
    if (fabs(d0[c]) < fabs(d0[ax])) ax = c;
  double a[3] = {0.0, 0.0, 0.0}, b1[3], b2[3];
  a[ax] = 1.0;
  cross3(a, d0, b1);
  normalize3(b1);
  cross3(d0, b1, b2);
  double al = 0.0, be = 0.0;
  int lit = 0, k = 0;
  double u[3] = {d0[0], d0[1], d0[2]}, cosg = 0.0;
  for (k = 0;; k++) {
    double d[3], e[3];
    for (int c = 0; c < 3; c++) d[c] = d0[c] + al * b1[c] + be * b2[c];
    normalize3(d);
    if (!shoot(m, sc, lt, integrator, q, d, e, u, 0, NULL)) break;
    double en = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    if (en <= lt->tol) { lit = 1; break; }
    if (k == lt->iters) break;
    /* forward-difference Jacobian columns de/dalpha, de/dbeta */
    double Jc[2][3], ud[3];
    int ok = 1;
    for (int col = 0; col < 2 && ok; col++) {
      double dd[3], ee[3];
      double aa = al + (col == 0 ? lt->delta : 0.0), bb = be + (col == 1 ? lt->delta : 0.0);
      for (int c = 0; c < 3; c++) dd[c] = d0[c] + aa * b1[c] + bb * b2[c];
      normalize3(dd);
      ok = shoot(m, sc, lt, integrator, q, dd, ee, ud, 0, NULL);
      for (int c = 0; c < 3; c++) Jc[col][c] = (ee[c] - e[c]) / lt->delta;
    }
    if (!ok) break;
    /* Gauss-Newton: (J^T J) step = -J^T e, by Cramer's rule */
    double A00 = 0, A01 = 0, A11 = 0, r0 = 0, r1 = 0;
    for (int c = 0; c < 3; c++) {
      A00 += Jc[0][c] * Jc[0][c];
      A01 += Jc[0][c] * Jc[1][c];
      A11 += Jc[1][c] * Jc[1][c];
      r0 -= Jc[0][c] * e[c];
      r1 -= Jc[1][c] * e[c];
    }
    double det = A00 * A11 - A01 * A01;
    if (!(det > 1e-12 * (A00 * A11))) break;
    double s0 = (r0 * A11 - r1 * A01) / det, s1 = (A00 * r1 - A01 * r0) / det;
    double sn = sqrt(s0 * s0 + s1 * s1);
    if (sn > 0.25) { s0 *= 0.25 / sn; s1 *= 0.25 / sn; }
    al += s0;
    be += s1;
  }
  if (iters_out) *iters_out = k;
  if (lit) {
    /* Riemannian cosine between the normal and the initial g-unit tangent */
    double g[9], gi[9];
    or_metric_tensor(m, q, g);
    or_inverse_by_minors(g, gi);
    double nn = 0.0;
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) nn += n[i] * gi[3 * i + j] * n[j];
    cosg = (n[0] * u[0] + n[1] * u[1] + n[2] * u[2]) / sqrt(nn);
    if (!(cosg > 0.0)) lit = 0;
  }
  if (lit) {
    double d[3], e[3], uu[3];
    for (int c = 0; c < 3; c++) d[c] = d0[c] + al * b1[c] + be * b2[c];
    normalize3(d);
    int blocked = 0;
    shoot(m, sc, lt, integrator, q, d, e, uu, 1, &blocked);
    if (blocked) lit = 0;
  }
  if (cos_out) *cos_out = cosg;
  if (u_out)
    for (int c = 0; c < 3; c++) u_out[c] = u[c];
  double inten = lit ? 0.1 + 0.9 * cosg : 0.1;
  for (int c = 0; c < 3; c++) {
    double v = sc->alb[3 * obj + c] * inten;
    v = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
    rgba[c] = (uint8_t)floor(255.0 * v + 0.5);
  }
  rgba[3] = 255;
  return lit;
}
