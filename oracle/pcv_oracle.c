/*
 * pcv_oracle.c -- plain FP64 CPU oracle for the path-CV / MSD hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs may load this code.  It shares nothing with the CUDA
 * library: no headers, no helpers, no constants.
 *
 * It follows Pazurikova et al., "Acceleration of Mean Square Distance Calculations
 * with Floating Close Structure in Metadynamics Simulations" (arXiv:1801.02362):
 *   - centring by the weighted centre (Section 3, first paragraph);
 *   - optimal rotation by the quaternion method of Kearsley / Coutsias (Section 3):
 *     the 4x4 symmetric matrix built from the 3x3 correlation matrix, its largest
 *     eigenvalue and eigenvector, here found by cyclic Jacobi rotations;
 *   - exact MSD, Eq. (dist), and its derivative, Eq. (der_dist), Algorithm 1;
 *   - property-map / path CV s, Eq. (property_map_cv), with q_i = i (1-based); the
 *     companion z = -(1/lambda) ln sum_i exp(-lambda D_i) of Branduardi et al. 2007,
 *     cited in Section 2;
 *   - floating close structure, Algorithm 2 with Eq. (close_dist) and
 *     Eq. (close_der_dist); refresh when D(x, y) > eps (strictly), y <- x (Section 3.2);
 *   - the neighbour list (Section 2, Section 3.1 after Eq. der_dist, the end of Section
 *     3.2, Section 6.2): every L steps the distances to all landmarks are computed and
 *     the M_nl closest kept; the other steps use only those.  With the close structure
 *     the list is chosen from the approximate distances, and a reassignment (which
 *     computes every distance exactly) also chooses it;
 *   - Gaussian-hill metadynamics bias on (s, z), Eq. (vbias), and its force through the
 *     path-CV derivatives;
 *   - cost model of Section 6.2 ("Theoretical Speedup") and Amdahl's law, Eq. (ahmdal).
 *
 * Everything is double precision, plain loops.  OpenMP threads share out independent
 * work only (frames of the exact-mode loop; within a frame the landmarks, then the atoms,
 * each output summed in the same order as a single thread would), so the results do not
 * depend on the thread count.
 * Conventions: coordinates are row-major (structure, atom, xyz).  R is row-major 3x3.
 * Two weight sets (Section 3.1, after Eq. der_dist): displacement weights w, the
 * contribution of each atom's displacement to the distance, and alignment weights w', the
 * contribution to the centre of mass that sets the translation.  Structures are centred by
 * their w'-weighted centres; R_{a x} maps the centred landmark a onto the centred frame x
 * minimising the distance itself, sum_j w_j |x_j - R a_j|^2 (the fit minimises the
 * distance, Section 3).  Both sets are normalised to sum 1; w' defaults to w.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOCONV -4

/* ------------------------------------------------------------------------------ */
/* small linear algebra                                                             */

/* weighted centre c = sum_j w_j x_j (w sums to 1) */
void orc_centroid(int n, const double* w, const double* x, double* c) {
  c[0] = c[1] = c[2] = 0.0;
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < 3; ++k) c[k] += w[j] * x[3 * j + k];
}

/* out = x - centre(x) */
void orc_center(int n, const double* w, const double* x, double* out) {
  double c[3];
  orc_centroid(n, w, x, c);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < 3; ++k) out[3 * j + k] = x[3 * j + k] - c[k];
}

/* The 4x4 symmetric quaternion matrix K of H (H[b][c] = sum_j w_j a_jb x_jc) such that
 * q^T K q = trace(R(q) H) for a unit quaternion q (Kearsley 1989 / Coutsias 2004). */
void orc_quat_matrix(const double* H, double* K) {
  const double hxx = H[0], hxy = H[1], hxz = H[2];
  const double hyx = H[3], hyy = H[4], hyz = H[5];
  const double hzx = H[6], hzy = H[7], hzz = H[8];
  K[0] = hxx + hyy + hzz;
  K[1] = hyz - hzy;
  K[2] = hzx - hxz;
  K[3] = hxy - hyx;
  K[5] = hxx - hyy - hzz;
  K[6] = hxy + hyx;
  K[7] = hzx + hxz;
  K[10] = -hxx + hyy - hzz;
  K[11] = hyz + hzy;
  K[15] = -hxx - hyy + hzz;
  K[4] = K[1];
  K[8] = K[2];
  K[9] = K[6];
  K[12] = K[3];
  K[13] = K[7];
  K[14] = K[11];
}

/* Rotation matrix of quaternion q = (s, v), normalised by |q|^2:
 * R = ((s^2 - |v|^2) I + 2 v v^T + 2 s [v]_x) / |q|^2 */
void orc_quat_to_rot(const double* q, double* R) {
  const double s = q[0], x = q[1], y = q[2], z = q[3];
  const double n2 = s * s + x * x + y * y + z * z;
  R[0] = (s * s + x * x - y * y - z * z) / n2;
  R[1] = 2.0 * (x * y - s * z) / n2;
  R[2] = 2.0 * (x * z + s * y) / n2;
  R[3] = 2.0 * (x * y + s * z) / n2;
  R[4] = (s * s - x * x + y * y - z * z) / n2;
  R[5] = 2.0 * (y * z - s * x) / n2;
  R[6] = 2.0 * (x * z - s * y) / n2;
  R[7] = 2.0 * (y * z + s * x) / n2;
  R[8] = (s * s - x * x - y * y + z * z) / n2;
}

/* Cyclic Jacobi eigen-solver for a symmetric 4x4 matrix.  On return evals[0..3] are
 * sorted in descending order and column k of evecs (evecs[4*i + k]) is the unit
 * eigenvector of evals[k].  Returns the number of sweeps, or -1 if 60 sweeps did not
 * bring the off-diagonal norm below 1e-15 of the diagonal's.  That stopping rule sits at the
 * FP64 rounding floor: the eigenvalues are then exact to ~1e-30 relative (second order in
 * the off-diagonal part), and the eigenvectors are exact up to mixing within a nearly
 * degenerate eigenspace, where every vector is optimal.  A stricter rule cannot be met when
 * the top eigenvalue is (nearly) double, e.g. for collinear structures. */
int orc_jacobi4(const double* Kin, double* evals, double* evecs) {
  double A[4][4], V[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      A[i][j] = Kin[4 * i + j];
      V[i][j] = (i == j) ? 1.0 : 0.0;
    }
  int sweep = 0, converged = 0;
  for (sweep = 1; sweep <= 60; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < 4; ++i) {
      diag += A[i][i] * A[i][i];
      for (int j = i + 1; j < 4; ++j) off += A[i][j] * A[i][j];
    }
    if (off == 0.0 || off <= 1e-30 * diag) {
      converged = 1;
      break;
    }
    for (int p = 0; p < 3; ++p)
      for (int r = p + 1; r < 4; ++r) {
        const double apr = A[p][r];
        if (apr == 0.0) continue;
        /* choose t = tan(phi) so that the rotated A[p][r] vanishes */
        const double theta = (A[r][r] - A[p][p]) / (2.0 * apr);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0);
        const double s = t * c;
        for (int k = 0; k < 4; ++k) { /* A <- A J  (columns p, r) */
          const double akp = A[k][p], akr = A[k][r];
          A[k][p] = c * akp - s * akr;
          A[k][r] = s * akp + c * akr;
        }
        for (int k = 0; k < 4; ++k) { /* A <- J^T A  (rows p, r) */
          const double apk = A[p][k], ark = A[r][k];
          A[p][k] = c * apk - s * ark;
          A[r][k] = s * apk + c * ark;
        }
        for (int k = 0; k < 4; ++k) { /* V <- V J */
          const double vkp = V[k][p], vkr = V[k][r];
          V[k][p] = c * vkp - s * vkr;
          V[k][r] = s * vkp + c * vkr;
        }
      }
  }
  int order[4] = {0, 1, 2, 3};
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j)
      if (A[order[j]][order[j]] > A[order[i]][order[i]]) {
        int tmp = order[i];
        order[i] = order[j];
        order[j] = tmp;
      }
  for (int k = 0; k < 4; ++k) {
    evals[k] = A[order[k]][order[k]];
    for (int i = 0; i < 4; ++i) evecs[4 * i + k] = V[i][order[k]];
  }
  return converged ? sweep : -1;
}

/* ------------------------------------------------------------------------------ */
/* one optimal superposition                                                        */

typedef struct {
  double D;          /* sum_j w_j |x_j - R a_j|^2, evaluated directly (Eq. dist) */
  double D_formula;  /* G_x + G_a - 2 lambda_max                                  */
  double Gx, Ga;     /* sum_j w_j |x_j|^2, sum_j w_j |a_j|^2 (centred)            */
  double R[9];       /* R_{a x}: rotation fitting a onto x                        */
  double q[4];       /* unit quaternion of R (sign: q[0] >= 0)                    */
  double evals[4];   /* eigenvalues of K, descending                              */
  double evecs[16];  /* eigenvectors of K (columns)                               */
  double H[9];       /* H[b][c] = sum_j w_j a_jb x_jc                             */
  int sweeps;
} orc_align_t;

/* Superimpose the already-centred structure a onto the already-centred x. */
int orc_align_centered(int n, const double* w, const double* x, const double* a, orc_align_t* o) {
  double H[9] = {0};
  double gx = 0.0, ga = 0.0;
  for (int j = 0; j < n; ++j) {
    const double* xj = x + 3 * j;
    const double* aj = a + 3 * j;
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) H[3 * b + c] += w[j] * aj[b] * xj[c];
    gx += w[j] * (xj[0] * xj[0] + xj[1] * xj[1] + xj[2] * xj[2]);
    ga += w[j] * (aj[0] * aj[0] + aj[1] * aj[1] + aj[2] * aj[2]);
  }
  double K[16];
  orc_quat_matrix(H, K);
  o->sweeps = orc_jacobi4(K, o->evals, o->evecs);
  for (int i = 0; i < 4; ++i) o->q[i] = o->evecs[4 * i + 0];
  if (o->q[0] < 0.0)
    for (int i = 0; i < 4; ++i) o->q[i] = -o->q[i];
  orc_quat_to_rot(o->q, o->R);
  memcpy(o->H, H, sizeof(H));
  o->Gx = gx;
  o->Ga = ga;
  o->D_formula = gx + ga - 2.0 * o->evals[0];
  double d = 0.0;
  for (int j = 0; j < n; ++j) {
    const double* xj = x + 3 * j;
    const double* aj = a + 3 * j;
    for (int b = 0; b < 3; ++b) {
      const double r = xj[b] - (o->R[3 * b + 0] * aj[0] + o->R[3 * b + 1] * aj[1] + o->R[3 * b + 2] * aj[2]);
      d += w[j] * r * r;
    }
  }
  o->D = d;
  return o->sweeps < 0 ? ORC_ENOCONV : ORC_OK;
}

/* Superimpose a onto x, both given uncentred. */
int orc_align(int n, const double* w, const double* x, const double* a, orc_align_t* o) {
  double* xc = (double*)malloc(sizeof(double) * 3 * n);
  double* ac = (double*)malloc(sizeof(double) * 3 * n);
  orc_center(n, w, x, xc);
  orc_center(n, w, a, ac);
  int st = orc_align_centered(n, w, xc, ac, o);
  free(xc);
  free(ac);
  return st;
}

/* Flat wrapper for foreign callers: out = [D, D_formula, Gx, Ga, R(9), q(4), evals(4),
 * evecs(16), H(9), sweeps] = 47 doubles. */
int orc_align_flat(int n, const double* w, const double* x, const double* a, double* out) {
  orc_align_t o;
  int st = orc_align(n, w, x, a, &o);
  out[0] = o.D;
  out[1] = o.D_formula;
  out[2] = o.Gx;
  out[3] = o.Ga;
  memcpy(out + 4, o.R, 9 * sizeof(double));
  memcpy(out + 13, o.q, 4 * sizeof(double));
  memcpy(out + 17, o.evals, 4 * sizeof(double));
  memcpy(out + 21, o.evecs, 16 * sizeof(double));
  memcpy(out + 37, o.H, 9 * sizeof(double));
  out[46] = (double)o.sweeps;
  return st;
}

/* ------------------------------------------------------------------------------ */
/* path collective variables                                                        */

/* s = sum q_i e_i / sum e_i and z = -(1/lambda) ln sum e_i with e_i = exp(-lambda D_i),
 * both evaluated with the shift m = min_i D_i.  p (optional) = e_i / sum e. */
void orc_path_cv(int m, const double* D, const double* qprop, double lambda, double* s,
                 double* z, double* p) {
  double dmin = D[0];
  for (int i = 1; i < m; ++i)
    if (D[i] < dmin) dmin = D[i];
  double l = 0.0, sq = 0.0;
  for (int i = 0; i < m; ++i) {
    const double e = exp(-lambda * (D[i] - dmin));
    l += e;
    sq += qprop[i] * e;
  }
  *s = sq / l;
  *z = dmin - log(l) / lambda;
  if (p)
    for (int i = 0; i < m; ++i) p[i] = exp(-lambda * (D[i] - dmin)) / l;
}

/* ------------------------------------------------------------------------------ */
/* per-frame evaluation                                                             */

static void normalise_weights(int n, const double* w_in, double* w) {
  if (!w_in) {
    for (int j = 0; j < n; ++j) w[j] = 1.0 / n;
    return;
  }
  double sum = 0.0;
  for (int j = 0; j < n; ++j) sum += w_in[j];
  for (int j = 0; j < n; ++j) w[j] = w_in[j] / sum;
}

/* Derivative of R(q) along dq for a unit quaternion q (dq orthogonal to q):
 * dR = 2 (s ds - v.dv) I + 2 (dv v^T + v dv^T) + 2 ds [v]_x + 2 s [dv]_x */
static void rot_differential(const double* q, const double* dq, double* dR) {
  const double s = q[0], v[3] = {q[1], q[2], q[3]};
  const double ds = dq[0], dv[3] = {dq[1], dq[2], dq[3]};
  const double diag = 2.0 * (s * ds - (v[0] * dv[0] + v[1] * dv[1] + v[2] * dv[2]));
  for (int b = 0; b < 3; ++b)
    for (int c = 0; c < 3; ++c) dR[3 * b + c] = (b == c ? diag : 0.0) + 2.0 * (dv[b] * v[c] + v[b] * dv[c]);
  /* [u]_x = [[0,-u3,u2],[u3,0,-u1],[-u2,u1,0]] */
  const double u[3] = {2.0 * (ds * v[0] + s * dv[0]), 2.0 * (ds * v[1] + s * dv[1]), 2.0 * (ds * v[2] + s * dv[2])};
  dR[1] -= u[2];
  dR[2] += u[1];
  dR[3] += u[2];
  dR[5] -= u[0];
  dR[6] -= u[1];
  dR[7] += u[0];
}

/* dR_{y x}/dx_{kc} for the rotation R fitting the centred y onto the centred x, from
 * first-order eigenvector perturbation of K: dq0 = sum_{l=1..3} v_l (v_l^T dK q0)/(l0 - l_l),
 * with dK = K(dH) and dH = d/dx_{kc} sum_j w_j y_j (x_j - centre(x))^T, the centre being
 * the w'-weighted one: dH = (w_k y_k - w'_k sum_j w_j y_j) e_c^T. */
static void rot_derivative_wrt_x(int n, const double* w, const double* wa, const double* yc, const orc_align_t* al,
                                 int k, int c, double* dR) {
  double ybar[3];
  orc_centroid(n, w, yc, ybar); /* sum_j w_j y_j */
  double dH[9] = {0};
  for (int b = 0; b < 3; ++b) dH[3 * b + c] = w[k] * yc[3 * k + b] - wa[k] * ybar[b];
  double dK[16];
  orc_quat_matrix(dH, dK);
  double q0[4];
  for (int i = 0; i < 4; ++i) q0[i] = al->evecs[4 * i + 0];
  double dKq[4];
  for (int i = 0; i < 4; ++i) {
    dKq[i] = 0.0;
    for (int j = 0; j < 4; ++j) dKq[i] += dK[4 * i + j] * q0[j];
  }
  double dq[4] = {0, 0, 0, 0};
  for (int l = 1; l < 4; ++l) {
    double num = 0.0;
    for (int i = 0; i < 4; ++i) num += al->evecs[4 * i + l] * dKq[i];
    const double coef = num / (al->evals[0] - al->evals[l]);
    for (int i = 0; i < 4; ++i) dq[i] += coef * al->evecs[4 * i + l];
  }
  rot_differential(q0, dq, dR);
}

/* The landmarks a frame is evaluated against: all M (sel == NULL) or the msel entries of
 * the neighbour list sel.  Path CVs over the members only (the sums of Eq.
 * property_map_cv run over the list); D of a landmark outside the list is +infinity. */
static int member(const int* sel, int k) { return sel ? sel[k] : k; }

static void members_cv(int msel, const int* sel, const double* D, const double* qprop, double lambda,
                       double* s, double* z, double* p) {
  double* Dm = (double*)malloc(sizeof(double) * msel);
  double* qm = (double*)malloc(sizeof(double) * msel);
  for (int k = 0; k < msel; ++k) {
    Dm[k] = D[member(sel, k)];
    qm[k] = qprop[member(sel, k)];
  }
  orc_path_cv(msel, Dm, qm, lambda, s, z, p);
  free(qm);
  free(Dm);
}

/* Exact evaluation of one frame (Algorithm 1 over the landmarks of sel, or all).
 * xc: centred frame; lmc: centred landmarks (M x N x 3).  Outputs D (M), R (M x 9,
 * optional), s, z, and gradients ds/dx, dz/dx (N x 3, optional), Eq. (der_dist).
 * D_given (M, optional): distances that replace the computed ones where not NaN, before
 * s, z and the weights of the gradient are formed (the geometry stays the oracle's own);
 * used to evaluate the derivatives at another evaluation's distances. */
static void take_given(int m, const double* D_given, double* D) {
  if (D_given)
    for (int i = 0; i < m; ++i)
      if (!isnan(D_given[i])) D[i] = D_given[i];
}
int orc_frame_exact(int m, int n, const double* w, const double* wa, const double* xc, const double* lmc,
                    const double* qprop, double lambda, const int* sel, int msel, double* s, double* z,
                    double* D, double* Rout, double* dsdx, double* dzdx, const double* D_given) {
  int st = ORC_OK;
  if (!sel) msel = m;
  double* R = (double*)calloc((size_t)9 * m, sizeof(double));
  for (int i = 0; i < m; ++i) D[i] = INFINITY;
  /* the landmarks are independent: OpenMP threads take them in parallel */
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
  for (int k = 0; k < msel; ++k) {
    const int i = member(sel, k);
    orc_align_t al;
    if (orc_align_centered(n, w, xc, lmc + (size_t)i * n * 3, &al) != ORC_OK) bad = 1;
    D[i] = al.D;
    memcpy(R + 9 * i, al.R, sizeof(al.R));
  }
  if (bad) st = ORC_ENOCONV;
  take_given(m, D_given, D);
  double* p = (double*)malloc(sizeof(double) * msel);
  members_cv(msel, sel, D, qprop, lambda, s, z, p);
  if (dsdx || dzdx) {
    /* Eq. (der_dist): dD_i/dx_k = 2 w_k d_ik + w'_k sum_j (-2 w_j d_ij) + (rotation term),
     * d_ij = x_j - R_i a_ij.  With R optimal for D the rotation term vanishes (stationarity
     * of D in R); the centre term vanishes only when w' = w.  First the centre sums of every
     * landmark (independent landmarks), then each atom's derivative summed over the
     * landmarks in order (independent atoms). */
    double* dsum = (double*)calloc((size_t)3 * (msel > 0 ? msel : 1), sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
    for (int k0 = 0; k0 < msel; ++k0) {
      const int i = member(sel, k0);
      const double* a = lmc + (size_t)i * n * 3;
      const double* Ri = R + 9 * i;
      double* ds3 = dsum + 3 * k0;
      for (int j = 0; j < n; ++j)
        for (int b = 0; b < 3; ++b) {
          const double d = xc[3 * j + b] - (Ri[3 * b] * a[3 * j] + Ri[3 * b + 1] * a[3 * j + 1] + Ri[3 * b + 2] * a[3 * j + 2]);
          ds3[b] += -2.0 * w[j] * d;
        }
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; ++k) {
      double gsk[3] = {0, 0, 0}, gzk[3] = {0, 0, 0};
      for (int k0 = 0; k0 < msel; ++k0) {
        const int i = member(sel, k0);
        const double* a = lmc + (size_t)i * n * 3;
        const double* Ri = R + 9 * i;
        const double gs = -lambda * p[k0] * (qprop[i] - *s); /* ds/dD_i */
        const double gz = p[k0];                           /* dz/dD_i */
        for (int b = 0; b < 3; ++b) {
          const double d = xc[3 * k + b] - (Ri[3 * b] * a[3 * k] + Ri[3 * b + 1] * a[3 * k + 1] + Ri[3 * b + 2] * a[3 * k + 2]);
          const double dDi = 2.0 * w[k] * d + wa[k] * dsum[3 * k0 + b];
          gsk[b] += gs * dDi;
          gzk[b] += gz * dDi;
        }
      }
      for (int b = 0; b < 3; ++b) {
        if (dsdx) dsdx[3 * k + b] = gsk[b];
        if (dzdx) dzdx[3 * k + b] = gzk[b];
      }
    }
    free(dsum);
  }
  if (Rout) memcpy(Rout, R, sizeof(double) * 9 * m);
  free(p);
  free(R);
  return st;
}

/* Approximate evaluation of one frame against close structure yc with stored rotations
 * B_i = R_{a_i y} (Algorithm 2, "else" branch): D~_i, Eq. (close_dist), and its
 * derivative, Eq. (close_der_dist).  al: the alignment of yc onto xc (R_{x y}). */
int orc_frame_approx(int m, int n, const double* w, const double* wa, const double* xc, const double* yc,
                     const double* B, const double* lmc, const double* qprop, double lambda,
                     const orc_align_t* al, const int* sel, int msel, double* s, double* z, double* D,
                     double* dsdx, double* dzdx, const double* D_given) {
  const double* Rxy = al->R;
  if (!sel) msel = m;
  double* Q = (double*)calloc((size_t)9 * m, sizeof(double));
  for (int i = 0; i < m; ++i) D[i] = INFINITY;
  /* the landmarks are independent: OpenMP threads take them in parallel */
#pragma omp parallel for schedule(dynamic, 4)
  for (int k0 = 0; k0 < msel; ++k0) {
    const int i = member(sel, k0);
    const double* Bi = B + 9 * i;
    double* Qi = Q + 9 * i;
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c)
        Qi[3 * b + c] = Rxy[3 * b] * Bi[c] + Rxy[3 * b + 1] * Bi[3 + c] + Rxy[3 * b + 2] * Bi[6 + c];
    const double* a = lmc + (size_t)i * n * 3;
    double dd = 0.0;
    for (int j = 0; j < n; ++j)
      for (int b = 0; b < 3; ++b) {
        const double r = xc[3 * j + b] - (Qi[3 * b] * a[3 * j] + Qi[3 * b + 1] * a[3 * j + 1] + Qi[3 * b + 2] * a[3 * j + 2]);
        dd += w[j] * r * r;
      }
    D[i] = dd;
  }
  take_given(m, D_given, D);
  double* p = (double*)malloc(sizeof(double) * msel);
  members_cv(msel, sel, D, qprop, lambda, s, z, p);
  if (dsdx || dzdx) {
    /* Eq. (close_der_dist) with d~_ij = x_j - Q_i a_ij: the direct and centre terms as in
     * the exact case, plus the rotation term through R_xy.  First, per landmark
     * (independent landmarks), the centre sum and G_i = sum_j -2 w_j d~_ij (R_{a_i y} a_ij)^T;
     * then G^s, G^z summed over the landmarks in order; then each atom's derivative summed
     * over the landmarks in order, plus its rotation term (independent atoms). */
    const int ms = msel > 0 ? msel : 1;
    double* dsum = (double*)calloc((size_t)3 * ms, sizeof(double));
    double* Gi = (double*)calloc((size_t)9 * ms, sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
    for (int k0 = 0; k0 < msel; ++k0) {
      const int i = member(sel, k0);
      const double* a = lmc + (size_t)i * n * 3;
      const double* Qi = Q + 9 * i;
      const double* Bi = B + 9 * i;
      double* ds3 = dsum + 3 * k0;
      double* G = Gi + 9 * k0;
      for (int j = 0; j < n; ++j) {
        double bj[3], dt[3];
        for (int b = 0; b < 3; ++b) bj[b] = Bi[3 * b] * a[3 * j] + Bi[3 * b + 1] * a[3 * j + 1] + Bi[3 * b + 2] * a[3 * j + 2];
        for (int b = 0; b < 3; ++b) {
          dt[b] = xc[3 * j + b] - (Qi[3 * b] * a[3 * j] + Qi[3 * b + 1] * a[3 * j + 1] + Qi[3 * b + 2] * a[3 * j + 2]);
          ds3[b] += -2.0 * w[j] * dt[b];
        }
        for (int b = 0; b < 3; ++b)
          for (int c = 0; c < 3; ++c) G[3 * b + c] += -2.0 * w[j] * dt[b] * bj[c];
      }
    }
    double Gs[9] = {0}, Gz[9] = {0}; /* sum_i (dL/dD_i) G_i for L = s and L = z */
    for (int k0 = 0; k0 < msel; ++k0) {
      const int i = member(sel, k0);
      const double gs = -lambda * p[k0] * (qprop[i] - *s);
      const double gz = p[k0];
      for (int e = 0; e < 9; ++e) {
        Gs[e] += gs * Gi[9 * k0 + e];
        Gz[e] += gz * Gi[9 * k0 + e];
      }
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < n; ++k) {
      double gsk[3] = {0, 0, 0}, gzk[3] = {0, 0, 0};
      for (int k0 = 0; k0 < msel; ++k0) {
        const int i = member(sel, k0);
        const double* a = lmc + (size_t)i * n * 3;
        const double* Qi = Q + 9 * i;
        const double gs = -lambda * p[k0] * (qprop[i] - *s);
        const double gz = p[k0];
        for (int b = 0; b < 3; ++b) {
          const double dt = xc[3 * k + b] - (Qi[3 * b] * a[3 * k] + Qi[3 * b + 1] * a[3 * k + 1] + Qi[3 * b + 2] * a[3 * k + 2]);
          const double dDi = 2.0 * w[k] * dt + wa[k] * dsum[3 * k0 + b];
          gsk[b] += gs * dDi;
          gzk[b] += gz * dDi;
        }
      }
      /* rotation term: sum_ab G_ab dR_{x y,ab}/dx_kc for each component c */
      for (int c = 0; c < 3; ++c) {
        double dR[9];
        rot_derivative_wrt_x(n, w, wa, yc, al, k, c, dR);
        double ts = 0.0, tz = 0.0;
        for (int e = 0; e < 9; ++e) {
          ts += Gs[e] * dR[e];
          tz += Gz[e] * dR[e];
        }
        gsk[c] += ts;
        gzk[c] += tz;
      }
      for (int b = 0; b < 3; ++b) {
        if (dsdx) dsdx[3 * k + b] = gsk[b];
        if (dzdx) dzdx[3 * k + b] = gzk[b];
      }
    }
    free(Gi);
    free(dsum);
  }
  free(p);
  free(Q);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------ */
/* batch drivers                                                                    */

static double* centred_copy(int count, int n, const double* w, const double* src) {
  double* out = (double*)malloc(sizeof(double) * (size_t)count * n * 3);
  for (int s = 0; s < count; ++s) orc_center(n, w, src + (size_t)s * n * 3, out + (size_t)s * n * 3);
  return out;
}

static void default_props(int m, const double* q_in, double* q) {
  for (int i = 0; i < m; ++i) q[i] = q_in ? q_in[i] : (double)(i + 1);
}

/* Exact path CVs for F frames (Algorithm 1, all landmarks, no neighbour list).
 * frames F x N x 3, landmarks M x N x 3 (uncentred), w (N) or NULL for uniform, q (M)
 * or NULL for q_i = i.  D (F x M), dsdx, dzdx (F x N x 3) optional. */
int orc_exact(int f, int m, int n, const double* w_in, const double* wa_in, const double* frames, const double* lm,
              const double* q_in, double lambda, double* s, double* z, double* D, double* dsdx,
              double* dzdx) {
  if (f < 0 || m < 1 || n < 1 || !(lambda > 0.0)) return ORC_EINVAL;
  double* w = (double*)malloc(sizeof(double) * n);
  double* wa = (double*)malloc(sizeof(double) * n);
  double* q = (double*)malloc(sizeof(double) * m);
  normalise_weights(n, w_in, w);
  normalise_weights(n, wa_in ? wa_in : w_in, wa);
  default_props(m, q_in, q);
  double* lmc = centred_copy(m, n, wa, lm);
  int st = ORC_OK;
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < f; ++t) {
    double* xc = (double*)malloc(sizeof(double) * 3 * n);
    double* Dt = (double*)malloc(sizeof(double) * m);
    orc_center(n, wa, frames + (size_t)t * n * 3, xc);
    int st_t = orc_frame_exact(m, n, w, wa, xc, lmc, q, lambda, NULL, 0, s + t, z + t, Dt, NULL,
                               dsdx ? dsdx + (size_t)t * n * 3 : NULL, dzdx ? dzdx + (size_t)t * n * 3 : NULL, NULL);
    if (D) memcpy(D + (size_t)t * m, Dt, sizeof(double) * m);
    if (st_t != ORC_OK) {
#pragma omp critical
      st = st_t;
    }
    free(Dt);
    free(xc);
  }
  free(lmc);
  free(q);
  free(wa);
  free(w);
  return st;
}

/* State carried between calls.  ctr: [0] has_y, [1] frames (the step index of the next
 * frame), [2] x-y alignments, [3] landmark alignments (exact MSDs), [4] approximate MSDs,
 * [5] threshold refreshes, [6] initial assignments, [7] a neighbour list is held. */
enum { C_HAS_Y = 0, C_FRAMES, C_XY, C_LMALIGN, C_APPROX, C_REF_THR, C_REF_INIT, C_HAS_NL };

/* Neighbour list: the m_nl landmarks with the smallest distances D_i (ties to the lower
 * index), written to out in increasing landmark index. */
void orc_nl_select(int m, const double* D, int m_nl, int* out) {
  unsigned char* taken = (unsigned char*)calloc((size_t)m, 1);
  for (int k = 0; k < m_nl; ++k) {
    int best = -1;
    for (int i = 0; i < m; ++i)
      if (!taken[i] && (best < 0 || D[i] < D[best])) best = i;
    taken[best] = 1;
  }
  int c = 0;
  for (int i = 0; i < m; ++i)
    if (taken[i]) out[c++] = i;
  free(taken);
}

/* Is step `step` a neighbour-list update of the original method: every l_stride steps
 * from the first, or whenever no list is held yet. */
static int nl_update_step(int64_t step, int l_stride, const int64_t* ctr) {
  return !ctr[C_HAS_NL] || step % l_stride == 0;
}

/* Exact path CVs with a neighbour list (the original method of Section 6.2: distances to
 * all M landmarks every L steps, to the M_nl listed ones otherwise), frames in time order.
 * nl_state: m_nl landmark indices carried between calls; ctr as for orc_close (frames,
 * landmark alignments, has-list).  m_nl <= 0 or >= M: no list. */
int orc_exact_nl(int f, int m, int n, const double* w_in, const double* wa_in, const double* frames,
                 const double* lm, const double* q_in, double lambda, int m_nl, int l_stride, int* nl_state,
                 int64_t* ctr, double* s, double* z, double* D, double* dsdx, double* dzdx) {
  if (f < 0 || m < 1 || n < 1 || !(lambda > 0.0) || l_stride < 1) return ORC_EINVAL;
  const int use_nl = m_nl > 0 && m_nl < m;
  double* w = (double*)malloc(sizeof(double) * n);
  double* wa = (double*)malloc(sizeof(double) * n);
  double* q = (double*)malloc(sizeof(double) * m);
  normalise_weights(n, w_in, w);
  normalise_weights(n, wa_in ? wa_in : w_in, wa);
  default_props(m, q_in, q);
  double* lmc = centred_copy(m, n, wa, lm);
  double* xc = (double*)malloc(sizeof(double) * 3 * n);
  double* Dt = (double*)malloc(sizeof(double) * m);
  int st = ORC_OK;
  for (int t = 0; t < f; ++t) {
    orc_center(n, wa, frames + (size_t)t * n * 3, xc);
    const int update = !use_nl || nl_update_step(ctr[C_FRAMES], l_stride, ctr);
    const int* sel = update ? NULL : nl_state;
    const int msel = update ? m : m_nl;
    if (orc_frame_exact(m, n, w, wa, xc, lmc, q, lambda, sel, msel, s + t, z + t, Dt, NULL,
                        dsdx ? dsdx + (size_t)t * n * 3 : NULL, dzdx ? dzdx + (size_t)t * n * 3 : NULL,
                        NULL) != ORC_OK)
      st = ORC_ENOCONV;
    if (use_nl && update) {
      orc_nl_select(m, Dt, m_nl, nl_state);
      ctr[C_HAS_NL] = 1;
    }
    ctr[C_LMALIGN] += msel;
    ctr[C_FRAMES] += 1;
    if (D) memcpy(D + (size_t)t * m, Dt, sizeof(double) * m);
  }
  free(Dt);
  free(xc);
  free(lmc);
  free(q);
  free(wa);
  free(w);
  return st;
}

/* Floating close structure, Algorithm 2, frames in time order.
 * y_state: N x 3 centred close structure; B_state: M x 9 rotations R_{a_i y}.
 * refreshed[t]: 0 approximate, 1 refresh (D(x,y) > eps), 2 initial assignment.
 * dxy[t]: D(x_t, y) that decided frame t (-1 at an initial assignment).
 * Neighbour list (m_nl in 1..M-1, else none): at a reassignment every distance is exact
 * and the list is chosen from them; at the other update steps (every l_stride steps) the
 * distances to all landmarks are the approximate ones of Eq. (close_dist) and the list is
 * chosen from those (end of Section 3.2); in between only the listed landmarks are
 * evaluated.  nl_state: m_nl indices carried between calls.
 * D_in (F x M, optional): distances that replace the frame's own (where not NaN) before
 * s, z and the derivative weights are formed; the decisions, rotations and geometry of the
 * derivatives stay the oracle's.  It evaluates the derivatives at another evaluation's
 * distances, which separates the error of a derivative computation from that of the
 * distances it was given. */
int orc_close(int f, int m, int n, const double* w_in, const double* wa_in, const double* frames, const double* lm,
              const double* q_in, double lambda, double eps, double* y_state, double* B_state,
              int m_nl, int l_stride, int* nl_state, int64_t* ctr, double* s, double* z, double* D,
              uint8_t* refreshed, double* dxy, double* dsdx, double* dzdx, const double* D_in) {
  if (f < 0 || m < 1 || n < 1 || !(lambda > 0.0) || !(eps >= 0.0) || l_stride < 1) return ORC_EINVAL;
  const int use_nl = m_nl > 0 && m_nl < m;
  double* w = (double*)malloc(sizeof(double) * n);
  double* q = (double*)malloc(sizeof(double) * m);
  double* wa = (double*)malloc(sizeof(double) * n);
  normalise_weights(n, w_in, w);
  normalise_weights(n, wa_in ? wa_in : w_in, wa);
  default_props(m, q_in, q);
  double* lmc = centred_copy(m, n, wa, lm);
  double* xc = (double*)malloc(sizeof(double) * 3 * n);
  double* Dt = (double*)malloc(sizeof(double) * m);
  double* Rt = (double*)malloc(sizeof(double) * 9 * m);
  int st = ORC_OK;
  for (int t = 0; t < f; ++t) {
    orc_center(n, wa, frames + (size_t)t * n * 3, xc);
    double* gs = dsdx ? dsdx + (size_t)t * n * 3 : NULL;
    double* gz = dzdx ? dzdx + (size_t)t * n * 3 : NULL;
    const double* Dg = D_in ? D_in + (size_t)t * m : NULL;
    int refresh = 0;
    orc_align_t al;
    if (!ctr[C_HAS_Y]) {
      refresh = 2;
      if (dxy) dxy[t] = -1.0;
    } else {
      /* R_xy, D(x, y) and (implicitly) dR_xy/dx: fit the close structure onto x */
      if (orc_align_centered(n, w, xc, y_state, &al) != ORC_OK) st = ORC_ENOCONV;
      ctr[C_XY] += 1;
      if (dxy) dxy[t] = al.D;
      if (al.D > eps) refresh = 1;
    }
    const int update = !use_nl || refresh || nl_update_step(ctr[C_FRAMES], l_stride, ctr);
    if (refresh) {
      /* reassign: exact distances to all landmarks, save R_{a_i x}, y <- x */
      if (orc_frame_exact(m, n, w, wa, xc, lmc, q, lambda, NULL, m, s + t, z + t, Dt, Rt, gs, gz, Dg) != ORC_OK)
        st = ORC_ENOCONV;
      memcpy(B_state, Rt, sizeof(double) * 9 * m);
      memcpy(y_state, xc, sizeof(double) * 3 * n);
      ctr[C_HAS_Y] = 1;
      ctr[C_LMALIGN] += m;
      ctr[refresh == 1 ? C_REF_THR : C_REF_INIT] += 1;
    } else {
      const int* sel = update ? NULL : nl_state;
      const int msel = update ? m : m_nl;
      orc_frame_approx(m, n, w, wa, xc, y_state, B_state, lmc, q, lambda, &al, sel, msel, s + t, z + t, Dt, gs, gz,
                       Dg);
      ctr[C_APPROX] += msel;
    }
    if (use_nl && update) {
      orc_nl_select(m, Dt, m_nl, nl_state);
      ctr[C_HAS_NL] = 1;
    }
    if (refreshed) refreshed[t] = (uint8_t)refresh;
    if (D) memcpy(D + (size_t)t * m, Dt, sizeof(double) * m);
    ctr[C_FRAMES] += 1;
  }
  free(Rt);
  free(Dt);
  free(xc);
  free(lmc);
  free(q);
  free(wa);
  free(w);
  return st;
}

/* Approximate distance of one frame to one landmark through a close structure, for
 * finite-difference checks: D~ = sum_j w_j |x_j - R_{x y} B a_j|^2 with x, y, a
 * uncentred on input. */
double orc_close_distance(int n, const double* w_in, const double* wa_in, const double* x, const double* y,
                          const double* B, const double* a) {
  double* w = (double*)malloc(sizeof(double) * n);
  double* wa = (double*)malloc(sizeof(double) * n);
  normalise_weights(n, w_in, w);
  normalise_weights(n, wa_in ? wa_in : w_in, wa);
  double* xc = (double*)malloc(sizeof(double) * 3 * n);
  double* yc = (double*)malloc(sizeof(double) * 3 * n);
  double* ac = (double*)malloc(sizeof(double) * 3 * n);
  orc_center(n, wa, x, xc);
  orc_center(n, wa, y, yc);
  orc_center(n, wa, a, ac);
  orc_align_t al;
  orc_align_centered(n, w, xc, yc, &al);
  double Q[9];
  for (int b = 0; b < 3; ++b)
    for (int c = 0; c < 3; ++c) Q[3 * b + c] = al.R[3 * b] * B[c] + al.R[3 * b + 1] * B[3 + c] + al.R[3 * b + 2] * B[6 + c];
  double dd = 0.0;
  for (int j = 0; j < n; ++j)
    for (int b = 0; b < 3; ++b) {
      const double r = xc[3 * j + b] - (Q[3 * b] * ac[3 * j] + Q[3 * b + 1] * ac[3 * j + 1] + Q[3 * b + 2] * ac[3 * j + 2]);
      dd += w[j] * r * r;
    }
  free(ac);
  free(yc);
  free(xc);
  free(wa);
  free(w);
  return dd;
}

/* ------------------------------------------------------------------------------ */
/* metadynamics bias on the path CVs, Eq. (vbias)                                   */

/* Gaussian-hill bias V(s, z) = sum_k w exp(-(s - s_k)^2 / (2 sigma_s^2) - (z - z_k)^2 /
 * (2 sigma_z^2)) over the hills deposited so far, and its derivatives dV/ds, dV/dz. */
void orc_hills_value(int n_hills, const double* hills, double w, double sigma_s, double sigma_z, double s, double z,
                     double* V, double* dVds, double* dVdz) {
  double v = 0.0, gs = 0.0, gz = 0.0;
  for (int k = 0; k < n_hills; ++k) {
    const double ds = s - hills[2 * k], dz = z - hills[2 * k + 1];
    const double e = w * exp(-ds * ds / (2.0 * sigma_s * sigma_s) - dz * dz / (2.0 * sigma_z * sigma_z));
    v += e;
    gs += -e * ds / (sigma_s * sigma_s);
    gz += -e * dz / (sigma_z * sigma_z);
  }
  *V = v;
  *dVds = gs;
  *dVdz = gz;
}

/* Metadynamics over F time-ordered frames with path CVs s, z and their derivatives (N x 3
 * per frame, optional).  Eq. (vbias) sums over the deposition times t' = tau_G, 2 tau_G, ...
 * that lie before t: steps are numbered from 0 (state[1] = steps done), a hill is deposited
 * at (s_t, z_t) after step t is evaluated when t is a positive multiple of the stride tau_G,
 * and step t sees the hills of the steps t' < t.  The first hill therefore lands at step
 * tau_G and the bias is zero up to and including that step.  Outputs V (F), and force =
 * -dV/dx = -(dV/ds ds/dx + dV/dz dz/dx) (F x N x 3, optional).  hills: capacity cap pairs
 * (s_k, z_k); state[0] = hills held.  Returns ORC_EINVAL when the capacity would be
 * exceeded. */
int orc_metad(int f, int n, const double* s, const double* z, const double* dsdx, const double* dzdx, double w,
              double sigma_s, double sigma_z, int stride, int cap, double* hills, int64_t* state, double* V,
              double* force) {
  if (f < 0 || n < 0 || stride < 1 || !(sigma_s > 0.0) || !(sigma_z > 0.0)) return ORC_EINVAL;
  for (int t = 0; t < f; ++t) {
    double dVds, dVdz;
    orc_hills_value((int)state[0], hills, w, sigma_s, sigma_z, s[t], z[t], V + t, &dVds, &dVdz);
    if (force && dsdx && dzdx)
      for (int e = 0; e < 3 * n; ++e)
        force[(size_t)t * 3 * n + e] = -(dVds * dsdx[(size_t)t * 3 * n + e] + dVdz * dzdx[(size_t)t * 3 * n + e]);
    if (state[1] > 0 && state[1] % stride == 0) {
      if (state[0] >= cap) return ORC_EINVAL;
      hills[2 * state[0]] = s[t];
      hills[2 * state[0] + 1] = z[t];
      state[0] += 1;
    }
    state[1] += 1;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------ */
/* cost model, Section 6.2 and Eq. (ahmdal)                                          */

/* Expensive distance computations per step, original method: M_nl + (N_ref - M_nl)/L
 * (no neighbour list: M_nl = 0, L = 1, giving N_ref). */
double orc_cost_original(double m_nl, double n_ref, double l_stride) { return m_nl + (n_ref - m_nl) / l_stride; }

/* Expensive distance computations per step with the close structure: 1 + N_ref/K. */
double orc_cost_close(double n_ref, double k_interval) { return 1.0 + n_ref / k_interval; }

/* Amdahl's law, Eq. (ahmdal): S = 1 / ((1 - p) + p/s). */
double orc_amdahl(double p, double s) { return 1.0 / ((1.0 - p) + p / s); }

/* Threads the OpenMP loops use (1 without OpenMP), and a way to set them (n >= 1). */
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
