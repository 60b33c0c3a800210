/*
 * FP64 CPU oracle for batched manifold projection and the sphere collision
 * check.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the CUDA path computes.  It is called by the tests, by
 * the package's smoke check and by the benchmark's CPU-baseline leg, never by
 * the product path.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * What it follows (paper: "Vectorizing Projection in Manifold-Constrained
 * Motion Planning for Real-Time Whole-Body Control"):
 *   - constraint residuals: TSR pose error Eq. 1 (Sec. II), the bimanual
 *     relative-pose error Eq. 2 (Sec. V-B), the humanoid's stacked feet /
 *     hands / centre-of-mass constraints (Sec. V-C, Fig. 6), with B^w = 0;
 *     the bounded TSR of Eq. 1 (distance outside the bounds B^w, Sec. II),
 *     point-on-plane and point-on-line task constraints (Sec. III) and the
 *     fixed distance of a closed linkage (Sec. V-C);
 *   - the SO(3) log map with a Taylor fallback of sinc near 0 (Sec. IV-A,
 *     "Tracing Compiler for Constraints");
 *   - ParallelProject and getDescentStep of Algorithm 2: d = F(q), stop when
 *     ||d|| < eps, otherwise q <- q - alpha J^T (J J^T + lambda I)^{-1} d,
 *     solved with a Cholesky factorisation (Sec. IV-A, "Vectorized
 *     Levenberg-Marquardt"), with the divergence exit on ||step|| >
 *     MaxDistance.  The stacked form uses all constraints in one step; the
 *     cyclic form (Sec. IV-C) takes one step per constraint in order.
 *   - the collision check as the definition: a configuration collides iff
 *     some robot sphere overlaps some obstacle sphere or box.
 *   - the projection's vector-Jacobian product at a point on the manifold:
 *     v = g - J^T (J J^T)^{-1} J g (the tangent-space projector).
 *   - ParallelConstrainedExtend of Algorithm 2: steer, project particles
 *     around q_steer (the earliest converged one wins), the 2 dist and r / n
 *     early exits, interpolation between q_s and q_proj, recursive bisection
 *     until the resolution is met, collision checks of every projected point.
 *
 * Conventions (shared with the input generators, not with the CUDA code):
 *   3x4 transforms are 12 doubles, row-major, column 3 = translation.
 *   T_j = T_parent(j) * X_j * Jnt(q_j); Jnt = Rz(q) (revolute) or Tz(q)
 *   (prismatic).  Batches are structure-of-arrays: q[j * ld + i].
 *
 * Every arithmetic function below is written out directly; the only library
 * calls are sqrt, sin, cos, atan2 from libm.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXJ 64
#define OR_MAXK 48
#define OR_MAXF 16
#define OR_MAXC 16

enum { OR_REVOLUTE = 0, OR_PRISMATIC = 1 };
enum {
  OR_SPHERE = 0, OR_AXIS_ALIGN = 1, OR_POSE = 2, OR_REL_POSE = 3, OR_COM_XY = 4,
  OR_PLANE = 5, OR_LINE = 6, OR_DIST = 7, OR_POSE_BOUNDED = 8, OR_COM_HULL = 9
};
enum {
  OR_CONVERGED = 1, OR_CAP = 2, OR_DIVERGED = 4, OR_NONFINITE = 8, OR_OUT_OF_LIMITS = 64
};

typedef struct {
  int32_t nj;
  const int32_t *parent;
  const int32_t *type;
  const double *X;        /* nj * 12 */
  const double *lower;
  const double *upper;
  const double *mass;     /* nj */
  const double *com;      /* nj * 3 */
  int32_t ns;
  const int32_t *sphere_link;
  const double *sphere;   /* ns * 4 */
  int32_t nf;
  const int32_t *frame_link;
  const double *frame_X;  /* nf * 12 */
} or_robot;

typedef struct {
  int32_t kind, fa, fb, pad;
  double P[12];
  double Q[12];
  double target[4];
  double B[12];   /* POSE_BOUNDED: lower[6] then upper[6] of [t; log R];
                     COM_HULL: the support polygon's vertices x0 y0 x1 y1 ..., counter-clockwise */
} or_constraint;

typedef struct {
  double tol;
  int32_t max_iters;
  int32_t cyclic;     /* 0: stacked F, one step per iteration; 1: cyclic over constraints */
  double lambda;
  double alpha;
  double max_step;    /* <= 0: divergence exit off */
  int32_t outer;      /* 0: inner form J^T (J J^T + lambda I)^{-1} F; 1: outer (J^T J + lambda I)^{-1} J^T F */
  int32_t pad;
} or_params;

/* ------------------------------------------------------------------------ */
/* 3x4 transforms                                                            */
/* ------------------------------------------------------------------------ */
static void tf_identity(double T[12]) {
  memset(T, 0, 12 * sizeof(double));
  T[0] = T[5] = T[10] = 1.0;
}

/* C = A * B (as 4x4 homogeneous matrices with last row 0 0 0 1). */
static void tf_mul(const double A[12], const double B[12], double C[12]) {
  double out[12];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 4; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[r * 4 + k] * B[k * 4 + c];
      if (c == 3) s += A[r * 4 + 3];
      out[r * 4 + c] = s;
    }
  }
  memcpy(C, out, sizeof(out));
}

/* Inverse of a rigid transform: [R^T, -R^T p]. */
static void tf_inv(const double A[12], double B[12]) {
  double out[12];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) out[r * 4 + c] = A[c * 4 + r];
    out[r * 4 + 3] = -(A[0 * 4 + r] * A[3] + A[1 * 4 + r] * A[7] + A[2 * 4 + r] * A[11]);
  }
  memcpy(B, out, sizeof(out));
}

static void tf_point(const double T[12], const double p[3], double out[3]) {
  double o[3];
  for (int r = 0; r < 3; ++r) o[r] = T[r * 4] * p[0] + T[r * 4 + 1] * p[1] + T[r * 4 + 2] * p[2] + T[r * 4 + 3];
  memcpy(out, o, sizeof(o));
}

/* out = R * v for the rotation part of T. */
static void tf_rotate(const double T[12], const double v[3], double out[3]) {
  double o[3];
  for (int r = 0; r < 3; ++r) o[r] = T[r * 4] * v[0] + T[r * 4 + 1] * v[1] + T[r * 4 + 2] * v[2];
  memcpy(out, o, sizeof(o));
}

/* out = R^T * v. */
static void tf_rotate_t(const double T[12], const double v[3], double out[3]) {
  double o[3];
  for (int r = 0; r < 3; ++r) o[r] = T[r] * v[0] + T[4 + r] * v[1] + T[8 + r] * v[2];
  memcpy(out, o, sizeof(o));
}

static void cross3(const double a[3], const double b[3], double out[3]) {
  double o[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  memcpy(out, o, sizeof(o));
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Joint motion: Rz(q) for revolute, translation q along z for prismatic. */
static void joint_motion(int type, double q, double M[12]) {
  tf_identity(M);
  if (type == OR_REVOLUTE) {
    double c = cos(q), s = sin(q);
    M[0] = c; M[1] = -s;
    M[4] = s; M[5] = c;
  } else {
    M[11] = q;
  }
}

/* ------------------------------------------------------------------------ */
/* Forward kinematics over the tree (paper Eq. 1: T_s^0 = FK(q)).            */
/* Tj[j]: world pose of joint frame j after its motion.                      */
/* z[j], o[j]: world axis and origin of joint j (frame T_parent * X_j).      */
/* ------------------------------------------------------------------------ */
typedef struct {
  double Tj[OR_MAXJ][12];
  double z[OR_MAXJ][3];
  double o[OR_MAXJ][3];
} or_kin;

static void fk(const or_robot *rb, const double *q, or_kin *K) {
  for (int j = 0; j < rb->nj; ++j) {
    double pre[12], M[12];
    if (rb->parent[j] < 0) memcpy(pre, rb->X + 12 * j, sizeof(pre));
    else tf_mul(K->Tj[rb->parent[j]], rb->X + 12 * j, pre);
    K->z[j][0] = pre[2]; K->z[j][1] = pre[6]; K->z[j][2] = pre[10];
    K->o[j][0] = pre[3]; K->o[j][1] = pre[7]; K->o[j][2] = pre[11];
    joint_motion(rb->type[j], q[j], M);
    tf_mul(pre, M, K->Tj[j]);
  }
}

static void frame_pose(const or_robot *rb, const or_kin *K, int f, double T[12]) {
  int link = rb->frame_link[f];
  if (link < 0) memcpy(T, rb->frame_X + 12 * f, 12 * sizeof(double));
  else tf_mul(K->Tj[link], rb->frame_X + 12 * f, T);
}

/* 1 if joint j lies on the path from the root to `link` (link itself included). */
static int is_ancestor(const or_robot *rb, int j, int link) {
  for (int l = link; l >= 0; l = rb->parent[l])
    if (l == j) return 1;
  return 0;
}

/* Velocity of a world point x under a unit rate of joint j (the world-frame
 * geometric Jacobian column): revolute z_j x (x - o_j), prismatic z_j. */
static void point_velocity(const or_robot *rb, const or_kin *K, int j, const double x[3], double v[3]) {
  if (rb->type[j] == OR_REVOLUTE) {
    double r[3] = {x[0] - K->o[j][0], x[1] - K->o[j][1], x[2] - K->o[j][2]};
    cross3(K->z[j], r, v);
  } else {
    v[0] = K->z[j][0]; v[1] = K->z[j][1]; v[2] = K->z[j][2];
  }
}

/* Angular velocity of downstream bodies under a unit rate of joint j. */
static void angular_velocity(const or_robot *rb, const or_kin *K, int j, double w[3]) {
  if (rb->type[j] == OR_REVOLUTE) { w[0] = K->z[j][0]; w[1] = K->z[j][1]; w[2] = K->z[j][2]; }
  else { w[0] = w[1] = w[2] = 0.0; }
}

/* ------------------------------------------------------------------------ */
/* SO(3) log map (Sec. IV-A).  theta = atan2(|w|, (tr R - 1) / 2) with       */
/* w = vee(R - R^T) / 2 = sin(theta) * axis.  Near theta = 0 the factor      */
/* theta / sin(theta) is replaced by its Taylor expansion 1 + theta^2 / 6.   */
/* Above 3*pi/4 the axis is read from the symmetric part                     */
/* (R + R^T) / 2 = cos(theta) I + (1 - cos(theta)) a a^T, its sign from w.   */
/* ------------------------------------------------------------------------ */
static void so3_log(const double T[12], double phi[3], double *theta_out) {
  double R[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) R[r][c] = T[r * 4 + c];
  double w[3] = {0.5 * (R[2][1] - R[1][2]), 0.5 * (R[0][2] - R[2][0]), 0.5 * (R[1][0] - R[0][1])};
  double cth = 0.5 * (R[0][0] + R[1][1] + R[2][2] - 1.0);
  double sth = sqrt(dot3(w, w));
  double theta = atan2(sth, cth);
  if (theta < 1e-3) {
    double f = 1.0 + theta * theta / 6.0;
    phi[0] = f * w[0]; phi[1] = f * w[1]; phi[2] = f * w[2];
  } else if (theta <= 0.75 * M_PI) {
    double f = theta / sth;
    phi[0] = f * w[0]; phi[1] = f * w[1]; phi[2] = f * w[2];
  } else {
    double S[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) S[r][c] = 0.5 * (R[r][c] + R[c][r]);
    int i = 0;
    if (S[1][1] > S[i][i]) i = 1;
    if (S[2][2] > S[i][i]) i = 2;
    double one_m_c = 1.0 - cth;
    double ai = sqrt((S[i][i] - cth) / one_m_c);
    double a[3];
    for (int r = 0; r < 3; ++r) a[r] = (S[r][i] - (r == i ? cth : 0.0)) / one_m_c / ai;
    if (dot3(a, w) < 0.0) { a[0] = -a[0]; a[1] = -a[1]; a[2] = -a[2]; }
    phi[0] = theta * a[0]; phi[1] = theta * a[1]; phi[2] = theta * a[2];
  }
  if (theta_out) *theta_out = theta;
}

/* Inverse left Jacobian of SO(3):
 *   Jl^{-1}(phi) = I - 1/2 [phi]x + beta [phi]x^2,
 *   beta = 1/theta^2 - sin(theta) / (2 theta (1 - cos(theta))),
 * with the series beta = 1/12 + theta^2/720 for small theta.  It maps a
 * world-side (left) angular velocity to the rate of change of log(R). */
static void so3_left_jac_inv(const double phi[3], double M[3][3]) {
  double th2 = dot3(phi, phi);
  double th = sqrt(th2);
  double beta;
  if (th < 1e-2) beta = 1.0 / 12.0 + th2 / 720.0;
  else beta = 1.0 / th2 - sin(th) / (2.0 * th * (1.0 - cos(th)));
  double P[3][3] = {{0.0, -phi[2], phi[1]}, {phi[2], 0.0, -phi[0]}, {-phi[1], phi[0], 0.0}};
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) {
      double P2 = 0.0;
      for (int k = 0; k < 3; ++k) P2 += P[r][k] * P[k][c];
      M[r][c] = (r == c ? 1.0 : 0.0) - 0.5 * P[r][c] + beta * P2;
    }
  }
}

static void mat3_vec(double M[3][3], const double v[3], double out[3]) {
  double o[3];
  for (int r = 0; r < 3; ++r) o[r] = M[r][0] * v[0] + M[r][1] * v[1] + M[r][2] * v[2];
  memcpy(out, o, sizeof(o));
}

/* ------------------------------------------------------------------------ */
/* Constraint residuals and analytic Jacobians.                              */
/* J is row-major [k][nj] with the constraint's rows starting at row0.       */
/* ------------------------------------------------------------------------ */
static int cons_dim(int kind) {
  switch (kind) {
    case OR_SPHERE: return 1;
    case OR_AXIS_ALIGN: return 2;
    case OR_POSE: return 6;
    case OR_REL_POSE: return 6;
    case OR_COM_XY: return 2;
    case OR_PLANE: return 1;
    case OR_LINE: return 2;
    case OR_DIST: return 1;
    case OR_POSE_BOUNDED: return 6;
    case OR_COM_HULL: return 2;
  }
  return 0;
}

/* Centre of mass: x_com = sum_i m_i c_i / sum_i m_i, c_i = T_i * com_i. */
static double com_world(const or_robot *rb, const or_kin *K, double x[3], double ci[][3]) {
  double M = 0.0;
  x[0] = x[1] = x[2] = 0.0;
  for (int i = 0; i < rb->nj; ++i) {
    tf_point(K->Tj[i], rb->com + 3 * i, ci[i]);
    M += rb->mass[i];
    for (int r = 0; r < 3; ++r) x[r] += rb->mass[i] * ci[i][r];
  }
  for (int r = 0; r < 3; ++r) x[r] /= M;
  return M;
}

/* CoM xy Jacobian rows: d x_com / d q_j = (1/M) sum over links i below j of
 * m_i * (velocity of c_i). */
static void com_jacobian_xy(const or_robot *rb, const or_kin *K, double ci[][3], double M, double *J, int row0) {
  const int d = rb->nj;
  for (int j = 0; j < d; ++j) {
    double acc[3] = {0, 0, 0};
    for (int i = 0; i < d; ++i) {
      if (!is_ancestor(rb, j, i)) continue;
      double v[3];
      point_velocity(rb, K, j, ci[i], v);
      for (int r = 0; r < 3; ++r) acc[r] += rb->mass[i] * v[r];
    }
    J[row0 * d + j] = acc[0] / M;
    J[(row0 + 1) * d + j] = acc[1] / M;
  }
}

/* Residual of one constraint (and, if J != NULL, its Jacobian rows). */
static int cons_eval(const or_robot *rb, const or_constraint *c, const double *q, const or_kin *K,
                     double *F, double *J, int row0) {
  const int d = rb->nj;
  switch (c->kind) {
    case OR_SPHERE: {
      /* F(q) = ||q|| - r */
      double n2 = 0.0;
      for (int j = 0; j < d; ++j) n2 += q[j] * q[j];
      double n = sqrt(n2);
      F[0] = n - c->target[0];
      if (J)
        for (int j = 0; j < d; ++j) J[row0 * d + j] = q[j] / n;
      return 1;
    }
    case OR_AXIS_ALIGN: {
      /* frame z-axis parallel to world z: F = (z_a . e_x, z_a . e_y) */
      double Ta[12];
      frame_pose(rb, K, c->fa, Ta);
      double za[3] = {Ta[2], Ta[6], Ta[10]};
      F[0] = za[0];
      F[1] = za[1];
      if (J) {
        int link = rb->frame_link[c->fa];
        for (int j = 0; j < d; ++j) {
          double w[3] = {0, 0, 0}, dz[3] = {0, 0, 0};
          if (link >= 0 && is_ancestor(rb, j, link)) {
            angular_velocity(rb, K, j, w);
            cross3(w, za, dz);
          }
          J[row0 * d + j] = dz[0];
          J[(row0 + 1) * d + j] = dz[1];
        }
      }
      return 2;
    }
    case OR_POSE:
    case OR_POSE_BOUNDED: {
      /* Eq. 1: T_err = (T_w^0)^{-1} T_s^0 (T_e^w)^{-1}, d = [t_err; log(R_err)] */
      double Ta[12], Pinv[12], Qinv[12], tmp[12], Terr[12], phi[3];
      frame_pose(rb, K, c->fa, Ta);
      tf_inv(c->P, Pinv);
      tf_inv(c->Q, Qinv);
      tf_mul(Pinv, Ta, tmp);
      tf_mul(tmp, Qinv, Terr);
      so3_log(Terr, phi, NULL);
      F[0] = Terr[3]; F[1] = Terr[7]; F[2] = Terr[11];
      F[3] = phi[0]; F[4] = phi[1]; F[5] = phi[2];
      if (J) {
        /* x: world position of the error frame's origin, T_a * Q^{-1} */
        double TaQ[12];
        tf_mul(Ta, Qinv, TaQ);
        double x[3] = {TaQ[3], TaQ[7], TaQ[11]};
        double Jl[3][3];
        so3_left_jac_inv(phi, Jl);
        int link = rb->frame_link[c->fa];
        for (int j = 0; j < d; ++j) {
          double v[3] = {0, 0, 0}, w[3] = {0, 0, 0}, vt[3], wt[3], dphi[3];
          if (link >= 0 && is_ancestor(rb, j, link)) {
            point_velocity(rb, K, j, x, v);
            angular_velocity(rb, K, j, w);
          }
          tf_rotate_t(c->P, v, vt);   /* P_R^T v */
          tf_rotate_t(c->P, w, wt);
          mat3_vec(Jl, wt, dphi);
          for (int r = 0; r < 3; ++r) {
            J[(row0 + r) * d + j] = vt[r];
            J[(row0 + 3 + r) * d + j] = dphi[r];
          }
        }
      }
      if (c->kind == OR_POSE_BOUNDED) {
        /* bounded TSR: each component's distance outside [lower, upper];
         * inside the bounds the residual and its derivative are zero */
        for (int r = 0; r < 6; ++r) {
          double lo = c->B[r], hi = c->B[6 + r];
          if (F[r] < lo) F[r] -= lo;
          else if (F[r] > hi) F[r] -= hi;
          else {
            F[r] = 0.0;
            if (J)
              for (int j = 0; j < d; ++j) J[(row0 + r) * d + j] = 0.0;
          }
        }
      }
      return 6;
    }
    case OR_PLANE:
    case OR_LINE: {
      /* origin x of frame a on the xy-plane (PLANE: F = z of P^{-1} x) or on
       * the z-axis (LINE: F = (x, y) of P^{-1} x) of the task frame P */
      double Ta[12], Pinv[12], xl[3];
      frame_pose(rb, K, c->fa, Ta);
      double x[3] = {Ta[3], Ta[7], Ta[11]};
      tf_inv(c->P, Pinv);
      tf_point(Pinv, x, xl);
      const int rows = c->kind == OR_PLANE ? 1 : 2;
      if (c->kind == OR_PLANE) F[0] = xl[2];
      else { F[0] = xl[0]; F[1] = xl[1]; }
      if (J) {
        int link = rb->frame_link[c->fa];
        for (int j = 0; j < d; ++j) {
          double v[3] = {0, 0, 0}, vt[3];
          if (link >= 0 && is_ancestor(rb, j, link)) point_velocity(rb, K, j, x, v);
          tf_rotate_t(c->P, v, vt);
          if (c->kind == OR_PLANE) J[row0 * d + j] = vt[2];
          else { J[row0 * d + j] = vt[0]; J[(row0 + 1) * d + j] = vt[1]; }
        }
      }
      return rows;
    }
    case OR_DIST: {
      /* closed linkage: F = |x_b - x_a| - L for the origins of frames a and b */
      double Ta[12], Tb[12];
      frame_pose(rb, K, c->fa, Ta);
      frame_pose(rb, K, c->fb, Tb);
      double xa[3] = {Ta[3], Ta[7], Ta[11]}, xb[3] = {Tb[3], Tb[7], Tb[11]};
      double e[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
      double n = sqrt(dot3(e, e));
      F[0] = n - c->target[0];
      if (J) {
        double u[3] = {e[0] / n, e[1] / n, e[2] / n};
        int la = rb->frame_link[c->fa], lb = rb->frame_link[c->fb];
        for (int j = 0; j < d; ++j) {
          double va[3] = {0, 0, 0}, vb[3] = {0, 0, 0};
          if (la >= 0 && is_ancestor(rb, j, la)) point_velocity(rb, K, j, xa, va);
          if (lb >= 0 && is_ancestor(rb, j, lb)) point_velocity(rb, K, j, xb, vb);
          double dv[3] = {vb[0] - va[0], vb[1] - va[1], vb[2] - va[2]};
          J[row0 * d + j] = dot3(u, dv);
        }
      }
      return 1;
    }
    case OR_REL_POSE: {
      /* Eq. 2: T_err = T_ref^{-1} (T_left^{-1} T_right), d = [t_err; log(R_err)] */
      double Ta[12], Tb[12], Tainv[12], Trefinv[12], rel[12], Terr[12], phi[3];
      frame_pose(rb, K, c->fa, Ta);
      frame_pose(rb, K, c->fb, Tb);
      tf_inv(Ta, Tainv);
      tf_inv(c->P, Trefinv);
      tf_mul(Tainv, Tb, rel);
      tf_mul(Trefinv, rel, Terr);
      so3_log(Terr, phi, NULL);
      F[0] = Terr[3]; F[1] = Terr[7]; F[2] = Terr[11];
      F[3] = phi[0]; F[4] = phi[1]; F[5] = phi[2];
      if (J) {
        /* A unit rate of joint j moves T_b (if j is above b) and T_a (if above
         * a) by the same world twist; T_a^{-1} T_b changes by sign s_j of that
         * twist applied to T_b, with s_j = [j above b] - [j above a].
         * G = R_ref^T R_a^T maps world vectors into the error frame. */
        double pb[3] = {Tb[3], Tb[7], Tb[11]};
        double G[12];
        tf_mul(Trefinv, Tainv, G);
        double Jl[3][3];
        so3_left_jac_inv(phi, Jl);
        int la = rb->frame_link[c->fa], lb = rb->frame_link[c->fb];
        for (int j = 0; j < d; ++j) {
          double s = (lb >= 0 && is_ancestor(rb, j, lb) ? 1.0 : 0.0) - (la >= 0 && is_ancestor(rb, j, la) ? 1.0 : 0.0);
          double v[3] = {0, 0, 0}, w[3] = {0, 0, 0}, vt[3], wt[3], dphi[3];
          if (s != 0.0) {
            point_velocity(rb, K, j, pb, v);
            angular_velocity(rb, K, j, w);
          }
          tf_rotate(G, v, vt);
          tf_rotate(G, w, wt);
          mat3_vec(Jl, wt, dphi);
          for (int r = 0; r < 3; ++r) {
            J[(row0 + r) * d + j] = s * vt[r];
            J[(row0 + 3 + r) * d + j] = s * dphi[r];
          }
        }
      }
      return 6;
    }
    case OR_COM_XY: {
      /* Sec. V-C stability constraint with the support-polygon centre as target:
       * F = x_com^{xy} - c */
      double x[3], ci[OR_MAXJ][3];
      double M = com_world(rb, K, x, ci);
      F[0] = x[0] - c->target[0];
      F[1] = x[1] - c->target[1];
      if (J) com_jacobian_xy(rb, K, ci, M, J, row0);
      return 2;
    }
    case OR_COM_HULL: {
      /* Sec. V-C stability constraint as printed: the CoM's xy distance to the
       * support polygon, zero inside.  F = c - P(c), P the nearest point of the
       * polygon (an edge's interior point or a vertex); dF/dq = n n^T J_com on
       * an edge (n its normal), J_com at a vertex, 0 inside. */
      double x[3], ci[OR_MAXJ][3];
      double M = com_world(rb, K, x, ci);
      const int nv = (int)c->target[0];
      int inside = 1;
      for (int e = 0; e < nv; ++e) {
        const double *a = c->B + 2 * e, *b = c->B + 2 * ((e + 1) % nv);
        double cr = (b[0] - a[0]) * (x[1] - a[1]) - (b[1] - a[1]) * (x[0] - a[0]);
        if (cr < 0.0) inside = 0;
      }
      double px = x[0], py = x[1], nx = 0.0, ny = 0.0;
      int on_edge = 0;
      if (!inside) {
        double best = INFINITY;
        for (int e = 0; e < nv; ++e) {
          const double *a = c->B + 2 * e, *b = c->B + 2 * ((e + 1) % nv);
          double ex = b[0] - a[0], ey = b[1] - a[1];
          double t = ((x[0] - a[0]) * ex + (x[1] - a[1]) * ey) / (ex * ex + ey * ey);
          int interior = t > 0.0 && t < 1.0;
          if (t < 0.0) t = 0.0;
          if (t > 1.0) t = 1.0;
          double qx = a[0] + t * ex, qy = a[1] + t * ey;
          double dd = (x[0] - qx) * (x[0] - qx) + (x[1] - qy) * (x[1] - qy);
          if (dd < best) {
            best = dd;
            px = qx;
            py = qy;
            on_edge = interior;
            double el = sqrt(ex * ex + ey * ey);
            nx = ey / el;
            ny = -ex / el;
          }
        }
      }
      F[0] = x[0] - px;
      F[1] = x[1] - py;
      if (J) {
        com_jacobian_xy(rb, K, ci, M, J, row0);
        for (int j = 0; j < d; ++j) {
          double g0 = J[row0 * d + j], g1 = J[(row0 + 1) * d + j];
          if (inside) {
            g0 = g1 = 0.0;
          } else if (on_edge) {
            double s = nx * g0 + ny * g1;
            g0 = nx * s;
            g1 = ny * s;
          }
          J[row0 * d + j] = g0;
          J[(row0 + 1) * d + j] = g1;
        }
      }
      return 2;
    }
  }
  return 0;
}

/* Stacked residual and Jacobian of constraints [c0, c1) (Sec. IV-C). */
static int eval_stack(const or_robot *rb, const or_constraint *cons, int c0, int c1, const double *q,
                      double *F, double *J) {
  or_kin K;
  fk(rb, q, &K);
  int k = 0;
  for (int i = c0; i < c1; ++i) {
    /* each constraint writes its own rows; J row offsets are relative to c0 */
    k += cons_eval(rb, &cons[i], q, &K, F + k, J, k);
  }
  return k;
}

/* ------------------------------------------------------------------------ */
/* Cholesky factorisation A = L L^T (Dahlquist & Bjorck), no pivoting.       */
/* Returns 0 if a pivot is not positive.                                     */
/* ------------------------------------------------------------------------ */
static int cholesky(int n, const double *A, double *L) {
  memset(L, 0, (size_t)n * n * sizeof(double));
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0.0)) return 0;
    L[j * n + j] = sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / L[j * n + j];
    }
  }
  return 1;
}

/* Solve L L^T x = b. */
static void chol_solve(int n, const double *L, const double *b, double *x) {
  double y[OR_MAXK > OR_MAXJ ? OR_MAXK : OR_MAXJ];
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
    y[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
}

/* LM step of Alg. 2: dq = alpha J^T (J J^T + lambda I)^{-1} F.  0 if singular. */
static int lm_step(int k, int d, const double *J, const double *F, double lambda, double alpha, double *dq) {
  double A[OR_MAXK * OR_MAXK], L[OR_MAXK * OR_MAXK], y[OR_MAXK];
  for (int a = 0; a < k; ++a) {
    for (int b = 0; b < k; ++b) {
      double s = 0.0;
      for (int j = 0; j < d; ++j) s += J[a * d + j] * J[b * d + j];
      A[a * k + b] = s + (a == b ? lambda : 0.0);
    }
  }
  if (!cholesky(k, A, L)) return 0;
  chol_solve(k, L, F, y);
  for (int j = 0; j < d; ++j) {
    double s = 0.0;
    for (int a = 0; a < k; ++a) s += J[a * d + j] * y[a];
    dq[j] = alpha * s;
  }
  return 1;
}

/* Outer form of the LM step (Alg. 2, the alternative of getDescentStep):
 * dq = alpha (J^T J + lambda I)^{-1} J^T F, a d x d system.  0 if singular. */
static int lm_step_outer(int k, int d, const double *J, const double *F, double lambda, double alpha, double *dq) {
  double A[OR_MAXJ * OR_MAXJ], L[OR_MAXJ * OR_MAXJ], b[OR_MAXJ], z[OR_MAXJ];
  for (int i = 0; i < d; ++i) {
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int a = 0; a < k; ++a) s += J[a * d + i] * J[a * d + j];
      A[i * d + j] = s + (i == j ? lambda : 0.0);
    }
    double s = 0.0;
    for (int a = 0; a < k; ++a) s += J[a * d + i] * F[a];
    b[i] = s;
  }
  if (!cholesky(d, A, L)) return 0;
  chol_solve(d, L, b, z);
  for (int j = 0; j < d; ++j) dq[j] = alpha * z[j];
  return 1;
}

static int descent(const or_params *p, int k, int d, const double *J, const double *F, double *dq) {
  return p->outer ? lm_step_outer(k, d, J, F, p->lambda, p->alpha, dq) : lm_step(k, d, J, F, p->lambda, p->alpha, dq);
}

static double norm(int n, const double *v) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += v[i] * v[i];
  return sqrt(s);
}

static int all_finite(int n, const double *v) {
  for (int i = 0; i < n; ++i)
    if (!isfinite(v[i])) return 0;
  return 1;
}

/* ParallelProject for one configuration (per-configuration exit):
 *   loop: d = F(q); if ||d|| < tol -> converged; if it == cap -> stop;
 *         step = getDescentStep(q); if ||step|| > max_step -> diverged;
 *         q += step.
 * Returns flags; *iters = number of steps applied; *resid = ||F(q_final)||. */
static int project_one(const or_robot *rb, const or_constraint *cons, int nc, const or_params *p, double *q,
                       int *iters, double *resid) {
  const int d = rb->nj;
  double F[OR_MAXK], J[OR_MAXK * OR_MAXJ], dq[OR_MAXJ], q0[OR_MAXJ];
  int flags = 0, it = 0;
  int k = 0;
  for (int i = 0; i < nc; ++i) k += cons_dim(cons[i].kind);
  for (;; ++it) {
    eval_stack(rb, cons, 0, nc, q, F, NULL);
    double r = norm(k, F);
    *resid = r;
    if (!isfinite(r)) { flags |= OR_NONFINITE; break; }
    if (r < p->tol) { flags |= OR_CONVERGED; break; }
    if (it == p->max_iters) { flags |= OR_CAP; break; }
    memcpy(q0, q, d * sizeof(double));
    if (!p->cyclic) {
      eval_stack(rb, cons, 0, nc, q, F, J);
      if (!descent(p, k, d, J, F, dq)) { flags |= OR_NONFINITE; break; }
      for (int j = 0; j < d; ++j) q[j] -= dq[j];
    } else {
      /* getDescentStep: one LM step per constraint F_i, in order */
      int singular = 0;
      for (int i = 0; i < nc && !singular; ++i) {
        int ki = eval_stack(rb, cons, i, i + 1, q, F, J);
        if (!descent(p, ki, d, J, F, dq)) { singular = 1; break; }
        for (int j = 0; j < d; ++j) q[j] -= dq[j];
      }
      if (singular) { flags |= OR_NONFINITE; break; }
    }
    double step2 = 0.0;
    for (int j = 0; j < d; ++j) step2 += (q[j] - q0[j]) * (q[j] - q0[j]);
    if (!all_finite(d, q)) { flags |= OR_NONFINITE; break; }
    if (p->max_step > 0.0 && sqrt(step2) > p->max_step) {
      memcpy(q, q0, d * sizeof(double));
      flags |= OR_DIVERGED;
      break;
    }
  }
  for (int j = 0; j < d; ++j)
    if (q[j] < rb->lower[j] || q[j] > rb->upper[j]) { flags |= OR_OUT_OF_LIMITS; break; }
  *iters = it;
  return flags;
}

/* ------------------------------------------------------------------------ */
/* Collision check: the definition, all pairs, strict inequality.            */
/* margin: smallest | distance - clearance | over all pairs, used by tests   */
/* to exclude verdicts within a rounding band of contact.                    */
/* ------------------------------------------------------------------------ */
static int check_one(const or_robot *rb, const double *q, int n_obs, const double *obs, int n_box,
                     const double *box, double *margin) {
  or_kin K;
  fk(rb, q, &K);
  int hit = 0;
  double m = INFINITY;
  for (int s = 0; s < rb->ns; ++s) {
    double c[3];
    const double *sp = rb->sphere + 4 * s;
    int link = rb->sphere_link[s];
    if (link < 0) { c[0] = sp[0]; c[1] = sp[1]; c[2] = sp[2]; }
    else tf_point(K.Tj[link], sp, c);
    double rs = sp[3];
    for (int o = 0; o < n_obs; ++o) {
      const double *ob = obs + 4 * o;
      double dx = c[0] - ob[0], dy = c[1] - ob[1], dz = c[2] - ob[2];
      double d2 = dx * dx + dy * dy + dz * dz;
      double rr = rs + ob[3];
      if (d2 < rr * rr) hit = 1;
      double gap = fabs(sqrt(d2) - rr);
      if (gap < m) m = gap;
    }
    for (int b = 0; b < n_box; ++b) {
      const double *bx = box + 6 * b;
      double d2 = 0.0;
      for (int r = 0; r < 3; ++r) {
        double e = 0.0;
        if (c[r] < bx[r]) e = bx[r] - c[r];
        else if (c[r] > bx[3 + r]) e = c[r] - bx[3 + r];
        d2 += e * e;
      }
      if (d2 < rs * rs) hit = 1;
      double gap = fabs(sqrt(d2) - rs);
      if (gap < m) m = gap;
    }
  }
  if (margin) *margin = m;
  return hit;
}


/* ------------------------------------------------------------------------ */
/* ParallelConstrainedExtend (Algorithm 2) for one extension.               */
/* The particles and the interpolated points are projected one by one (each */
/* with its own exit); the lockstep early exits of the algorithm become:    */
/* the projection of the particles succeeds if some particle converges no   */
/* later than the first step that exceeds MaxDistance (the convergence test */
/* of an iteration precedes its step), and the winner is the particle that  */
/* converged after the fewest steps (lowest index on ties).                 */
/* ------------------------------------------------------------------------ */
enum {
  OR_EXT_OK = 0, OR_EXT_DEGENERATE = 1, OR_EXT_NO_PROJECTION = 2, OR_EXT_PROJ_COLLISION = 3, OR_EXT_TOO_FAR = 4,
  OR_EXT_INTERP_FAIL = 5, OR_EXT_GAP = 6, OR_EXT_INTERP_COLLISION = 7, OR_EXT_RESOLUTION = 8
};
#define OR_EXT_MAXN 32
#define OR_EXT_MAXPTS 128   /* points of the validated chain, both ends included */

typedef struct {
  double r;          /* extension range */
  double delta;      /* resolution: consecutive validated points at most delta apart */
  int32_t n;         /* particles = interpolated points (<= 32) */
  int32_t max_depth; /* bisection levels after the first interpolation */
} or_ext_params;

static double dist2(int d, const double *a, const double *b) {
  double s = 0.0;
  for (int j = 0; j < d; ++j) s += (a[j] - b[j]) * (a[j] - b[j]);
  return s;
}

typedef double or_pt[OR_MAXJ];

static int extend_body(const or_robot *rb, const or_constraint *cons, int nc, const or_params *p,
                       const or_ext_params *e, int n_obs, const double *obs, int n_box, const double *box,
                       const double *qs, const double *qt, const double *eps, double *q_proj, int *n_points,
                       int *winner, or_pt *chain, or_pt *next) {
  const int d = rb->nj, n = e->n;
  double v[OR_MAXJ], steer[OR_MAXJ], x[OR_MAXJ];
  *n_points = 0;
  *winner = -1;
  for (int j = 0; j < d; ++j) q_proj[j] = qs[j];
  double len = sqrt(dist2(d, qt, qs));
  if (!(len > 0.0)) return OR_EXT_DEGENERATE;
  double dist = len < e->r ? len : e->r;
  for (int j = 0; j < d; ++j) {
    v[j] = (qt[j] - qs[j]) / len;
    steer[j] = qs[j] + dist * v[j];
  }
  /* particles around q_steer along v; the earliest converged one */
  int best = -1, best_it = 1 << 30, first_div = 1 << 30;
  double qp[OR_MAXJ];
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < d; ++j) x[j] = steer[j] + eps[i] * v[j];
    int it = 0;
    double res = 0.0;
    int f = project_one(rb, cons, nc, p, x, &it, &res);
    if ((f & OR_CONVERGED) && it < best_it) {
      best = i;
      best_it = it;
      memcpy(qp, x, sizeof(double) * d);
    }
    if ((f & OR_DIVERGED) && it < first_div) first_div = it;
  }
  if (best < 0 || first_div < best_it) return OR_EXT_NO_PROJECTION;
  *winner = best;
  memcpy(q_proj, qp, sizeof(double) * d);
  *n_points = 1;
  if (check_one(rb, qp, n_obs, obs, n_box, box, NULL)) return OR_EXT_PROJ_COLLISION;
  if (sqrt(dist2(d, qp, qs)) > 2.0 * dist) return OR_EXT_TOO_FAR;
  /* n points between q_s and q_proj, projected; chain q_s, x_1 .. x_n, q_proj */
  int m = 0;
  memcpy(chain[m++], qs, sizeof(double) * d);
  for (int k = 1; k <= n; ++k) {
    double t = (double)k / (double)(n + 1);
    for (int j = 0; j < d; ++j) x[j] = qs[j] + t * (qp[j] - qs[j]);
    int it = 0;
    double res = 0.0;
    int f = project_one(rb, cons, nc, p, x, &it, &res);
    if (!(f & OR_CONVERGED)) return OR_EXT_INTERP_FAIL;
    memcpy(chain[m++], x, sizeof(double) * d);
  }
  memcpy(chain[m++], qp, sizeof(double) * d);
  *n_points += n;
  for (int k = 0; k + 1 < m; ++k)
    if (sqrt(dist2(d, chain[k], chain[k + 1])) > e->r / n) return OR_EXT_GAP;
  for (int k = 1; k + 1 < m; ++k)
    if (check_one(rb, chain[k], n_obs, obs, n_box, box, NULL)) return OR_EXT_INTERP_COLLISION;
  /* bisect every gap above the resolution, level by level: the midpoint's
   * projection must converge, split the gap into two no longer than it, and
   * be collision-free */
  for (int level = 0;; ++level) {
    int wide = 0;
    for (int k = 0; k + 1 < m; ++k)
      if (sqrt(dist2(d, chain[k], chain[k + 1])) > e->delta) ++wide;
    if (wide == 0) break;
    if (level >= e->max_depth || m + wide > OR_EXT_MAXPTS) return OR_EXT_RESOLUTION;
    int m2 = 0;
    for (int k = 0; k + 1 < m; ++k) {
      memcpy(next[m2++], chain[k], sizeof(double) * d);
      double g = sqrt(dist2(d, chain[k], chain[k + 1]));
      if (g > e->delta) {
        for (int j = 0; j < d; ++j) x[j] = 0.5 * (chain[k][j] + chain[k + 1][j]);
        int it = 0;
        double res = 0.0;
        int f = project_one(rb, cons, nc, p, x, &it, &res);
        if (!(f & OR_CONVERGED)) return OR_EXT_INTERP_FAIL;
        if (sqrt(dist2(d, chain[k], x)) > g || sqrt(dist2(d, x, chain[k + 1])) > g) return OR_EXT_GAP;
        if (check_one(rb, x, n_obs, obs, n_box, box, NULL)) return OR_EXT_INTERP_COLLISION;
        memcpy(next[m2++], x, sizeof(double) * d);
        *n_points += 1;
      }
    }
    memcpy(next[m2++], chain[m - 1], sizeof(double) * d);
    m = m2;
    memcpy(chain, next, sizeof(or_pt) * m);
  }
  return OR_EXT_OK;
}

static int extend_one(const or_robot *rb, const or_constraint *cons, int nc, const or_params *p,
                      const or_ext_params *e, int n_obs, const double *obs, int n_box, const double *box,
                      const double *qs, const double *qt, const double *eps, double *q_proj, int *n_points,
                      int *winner) {
  or_pt *buf = (or_pt *)malloc(sizeof(or_pt) * 2 * OR_EXT_MAXPTS);
  if (!buf) return OR_EXT_RESOLUTION;
  int st = extend_body(rb, cons, nc, p, e, n_obs, obs, n_box, box, qs, qt, eps, q_proj, n_points, winner, buf,
                       buf + OR_EXT_MAXPTS);
  free(buf);
  return st;
}

/* ------------------------------------------------------------------------ */
/* VJP of the projection at a point on the manifold:                         */
/*   v = g - J^T (J J^T)^{-1} J g.  Returns 0 if J J^T is singular.          */
/* ------------------------------------------------------------------------ */
static int vjp_one(const or_robot *rb, const or_constraint *cons, int nc, const double *q, const double *g,
                   double *v) {
  const int d = rb->nj;
  double F[OR_MAXK], J[OR_MAXK * OR_MAXJ], u[OR_MAXK], y[OR_MAXJ];
  int k = eval_stack(rb, cons, 0, nc, q, F, J);
  for (int a = 0; a < k; ++a) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) s += J[a * d + j] * g[j];
    u[a] = s;
  }
  if (!lm_step(k, d, J, u, 0.0, 1.0, y)) {
    for (int j = 0; j < d; ++j) v[j] = NAN;
    return 0;
  }
  for (int j = 0; j < d; ++j) v[j] = g[j] - y[j];
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Gradient path shortening on the manifold: the consumer of the VJP above   */
/* (the paper makes its log map differentiable so that the projection can   */
/* serve gradient-based optimisation, Sec. IV-A).                            */
/*                                                                           */
/* A path is n_way waypoints q_0 .. q_{n_way-1} (columns w of a d x n_way    */
/* block).  Its length is the sum of the Euclidean lengths of its edges,     */
/*   L = sum_{w=0}^{n_way-2} |q_{w+1} - q_w|,                                */
/* so dL/dq_w = e_w / |e_w| - e_{w+1} / |e_{w+1}| with e_w = q_w - q_{w-1}   */
/* (an edge that does not exist, or has zero length, contributes nothing).  */
/*                                                                           */
/* One descent step from the waypoints Q:                                    */
/*   1. P_w = project(Q_w) for every waypoint (ParallelProject above);       */
/*   2. G = dL/dP at the projected path;                                     */
/*   3. V_w = VJP(P_w, G_w) = G_w - J^T (J J^T)^{-1} J G_w, the gradient     */
/*      pulled back through the projection (its tangent component);         */
/*   4. Q_w = P_w - s_w eta V_w for the interior waypoints, where            */
/*      s_w = min(1, max_step / max_j |eta V_w[j]|) clips the largest joint  */
/*      move of a waypoint to max_step (max_step <= 0: no clipping); the     */
/*      endpoints stay at P_0 and P_{n_way-1}.                               */
/* After the last step the waypoints are projected once more.                */
/* ------------------------------------------------------------------------ */
static double path_length(int d, int n_way, const double *Q /* [n_way][d] */) {
  double L = 0.0;
  for (int w = 0; w + 1 < n_way; ++w) L += sqrt(dist2(d, Q + (w + 1) * d, Q + w * d));
  return L;
}

static void path_gradient(int d, int n_way, const double *Q, double *G) {
  for (int w = 0; w < n_way; ++w) {
    double *g = G + w * d;
    for (int j = 0; j < d; ++j) g[j] = 0.0;
    if (w > 0) {   /* the edge into q_w: + e_w / |e_w| */
      const double n = sqrt(dist2(d, Q + w * d, Q + (w - 1) * d));
      if (n > 0.0)
        for (int j = 0; j < d; ++j) g[j] += (Q[w * d + j] - Q[(w - 1) * d + j]) / n;
    }
    if (w + 1 < n_way) {   /* the edge out of q_w: - e_{w+1} / |e_{w+1}| */
      const double n = sqrt(dist2(d, Q + (w + 1) * d, Q + w * d));
      if (n > 0.0)
        for (int j = 0; j < d; ++j) g[j] -= (Q[(w + 1) * d + j] - Q[w * d + j]) / n;
    }
  }
}

/* Shortens one path in place (Q [n_way][d]): `steps` descent steps, then the
 * final projection.  L_out[0] = length of the input, L_out[1] = length of the
 * result; flags / resid of the final projection per waypoint.  Returns 0 if
 * the scratch could not be allocated. */
static int shorten_one(const or_robot *rb, const or_constraint *cons, int nc, const or_params *p, int n_way,
                       int steps, double eta, double max_step, double *Q, uint8_t *flags, double *resid,
                       double *L_out) {
  const int d = rb->nj;
  double *G = (double *)malloc(sizeof(double) * (size_t)n_way * d);
  if (!G) return 0;
  L_out[0] = path_length(d, n_way, Q);
  for (int s = 0; s <= steps; ++s) {
    for (int w = 0; w < n_way; ++w) {   /* 1. project every waypoint */
      int it = 0;
      double r = 0.0;
      int f = project_one(rb, cons, nc, p, Q + w * d, &it, &r);
      flags[w] = (uint8_t)f;
      resid[w] = r;
    }
    if (s == steps) break;   /* the final projection */
    path_gradient(d, n_way, Q, G);   /* 2. */
    for (int w = 1; w + 1 < n_way; ++w) {
      double v[OR_MAXJ];
      vjp_one(rb, cons, nc, Q + w * d, G + w * d, v);   /* 3. (NaN if J J^T is singular) */
      double m = 0.0;
      for (int j = 0; j < d; ++j) m = fmax(m, fabs(eta * v[j]));
      const double sc = (max_step > 0.0 && m > max_step) ? max_step / m : 1.0;
      for (int j = 0; j < d; ++j) Q[w * d + j] -= sc * eta * v[j];   /* 4. */
    }
  }
  L_out[1] = path_length(d, n_way, Q);
  free(G);
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Exported API (plain pointers; batches are SoA with leading dimension ld). */
/* ------------------------------------------------------------------------ */

/* World poses of every joint frame and of every task frame at q. */
void or_fk(const or_robot *rb, const double *q, double *Tj, double *Tf) {
  or_kin K;
  fk(rb, q, &K);
  if (Tj) memcpy(Tj, K.Tj, (size_t)rb->nj * 12 * sizeof(double));
  if (Tf)
    for (int f = 0; f < rb->nf; ++f) frame_pose(rb, &K, f, Tf + 12 * f);
}

/* Joint axes and origins (world) at q. */
void or_joint_axes(const or_robot *rb, const double *q, double *z, double *o) {
  or_kin K;
  fk(rb, q, &K);
  memcpy(z, K.z, (size_t)rb->nj * 3 * sizeof(double));
  memcpy(o, K.o, (size_t)rb->nj * 3 * sizeof(double));
}

/* Centre of mass at q. */
double or_com(const or_robot *rb, const double *q, double *x) {
  or_kin K;
  double ci[OR_MAXJ][3];
  fk(rb, q, &K);
  return com_world(rb, &K, x, ci);
}

/* Stacked residual F (k) and Jacobian J (k x nj, row-major) at q; J may be NULL. */
int or_residual_jacobian(const or_robot *rb, const or_constraint *cons, int nc, const double *q, double *F,
                         double *J) {
  return eval_stack(rb, cons, 0, nc, q, F, J);
}

void or_so3_log(const double *T, double *phi) { so3_log(T, phi, NULL); }
void or_so3_left_jac_inv(const double *phi, double *M) {
  double m[3][3];
  so3_left_jac_inv(phi, m);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) M[r * 3 + c] = m[r][c];
}

/* Fill constraint references from the robot's pose at q_ref (one config):
 *   POSE:     P := T_a(q_ref) Q^{-1}          (so that T_err(q_ref) = I)
 *   REL_POSE: P := T_a(q_ref)^{-1} T_b(q_ref)
 *   COM_XY:   target := xy midpoint of frames a and b at q_ref
 *             (the centre of the support polygon spanned by the two feet). */
void or_resolve_reference(const or_robot *rb, or_constraint *c, const double *q_ref) {
  or_kin K;
  fk(rb, q_ref, &K);
  if (c->kind == OR_POSE || c->kind == OR_POSE_BOUNDED) {
    double Ta[12], Qinv[12];
    frame_pose(rb, &K, c->fa, Ta);
    tf_inv(c->Q, Qinv);
    tf_mul(Ta, Qinv, c->P);
  } else if (c->kind == OR_PLANE || c->kind == OR_LINE) {
    /* the plane / line keeps its orientation and passes through frame a */
    double Ta[12];
    frame_pose(rb, &K, c->fa, Ta);
    c->P[3] = Ta[3];
    c->P[7] = Ta[7];
    c->P[11] = Ta[11];
  } else if (c->kind == OR_DIST) {
    double Ta[12], Tb[12];
    frame_pose(rb, &K, c->fa, Ta);
    frame_pose(rb, &K, c->fb, Tb);
    double e[3] = {Tb[3] - Ta[3], Tb[7] - Ta[7], Tb[11] - Ta[11]};
    c->target[0] = sqrt(dot3(e, e));
  } else if (c->kind == OR_REL_POSE) {
    double Ta[12], Tb[12], Tainv[12];
    frame_pose(rb, &K, c->fa, Ta);
    frame_pose(rb, &K, c->fb, Tb);
    tf_inv(Ta, Tainv);
    tf_mul(Tainv, Tb, c->P);
  } else if (c->kind == OR_COM_XY) {
    double Ta[12], Tb[12];
    frame_pose(rb, &K, c->fa, Ta);
    frame_pose(rb, &K, c->fb, Tb);
    c->target[0] = 0.5 * (Ta[3] + Tb[3]);
    c->target[1] = 0.5 * (Ta[7] + Tb[7]);
  } else if (c->kind == OR_COM_HULL) {
    /* the support polygon: the xy box around frames a and b grown by the
     * margin target[1], counter-clockwise */
    double Ta[12], Tb[12];
    frame_pose(rb, &K, c->fa, Ta);
    frame_pose(rb, &K, c->fb, Tb);
    double m = c->target[1];
    double x0 = fmin(Ta[3], Tb[3]) - m, x1 = fmax(Ta[3], Tb[3]) + m;
    double y0 = fmin(Ta[7], Tb[7]) - m, y1 = fmax(Ta[7], Tb[7]) + m;
    double v[8] = {x0, y0, x1, y0, x1, y1, x0, y1};
    memcpy(c->B, v, sizeof(v));
    c->target[0] = 4.0;
  }
}

typedef struct {
  const or_robot *rb;
  const or_constraint *cons;
  int nc;
  const or_params *p;
  int64_t i0, i1, ld;
  const double *q_in;
  double *q_out;
  uint8_t *flags;
  int32_t *iters;
  double *resid;
  /* check */
  int n_obs, n_box;
  const double *obs, *box;
  uint8_t *hit;
  double *margin;
  /* vjp */
  const double *g;
  double *v;
  /* extend */
  const or_ext_params *ep;
  const double *q_t, *eps;
  int64_t ld_eps;
  int32_t *n_points, *winner;
  /* path shortening: one job item is one path of n_way consecutive columns */
  int n_way, steps;
  double eta, max_step;
  double *lengths;   /* [n_paths][2]: before, after */
  int *failed;
  int mode;
} or_job;

static void *job_run(void *arg) {
  or_job *jb = (or_job *)arg;
  const int d = jb->rb->nj;
  double q[OR_MAXJ], g[OR_MAXJ], v[OR_MAXJ];
  for (int64_t i = jb->i0; i < jb->i1; ++i) {
    if (jb->mode != 4)
      for (int j = 0; j < d; ++j) q[j] = jb->q_in[j * jb->ld + i];
    if (jb->mode == 0) {
      int it = 0;
      double r = 0.0;
      int f = project_one(jb->rb, jb->cons, jb->nc, jb->p, q, &it, &r);
      for (int j = 0; j < d; ++j) jb->q_out[j * jb->ld + i] = q[j];
      jb->flags[i] = (uint8_t)f;
      jb->iters[i] = it;
      jb->resid[i] = r;
    } else if (jb->mode == 1) {
      double m = 0.0;
      jb->hit[i] = (uint8_t)check_one(jb->rb, q, jb->n_obs, jb->obs, jb->n_box, jb->box, &m);
      if (jb->margin) jb->margin[i] = m;
    } else if (jb->mode == 4) {
      /* path i: columns i * n_way .. (i + 1) * n_way - 1, gathered as [n_way][d] */
      const int nw = jb->n_way;
      double *Q = (double *)malloc(sizeof(double) * (size_t)nw * d);
      if (!Q) { *jb->failed = 1; continue; }
      const int64_t c0 = i * nw;
      for (int w = 0; w < nw; ++w)
        for (int j = 0; j < d; ++j) Q[w * d + j] = jb->q_in[j * jb->ld + c0 + w];
      if (!shorten_one(jb->rb, jb->cons, jb->nc, jb->p, nw, jb->steps, jb->eta, jb->max_step, Q,
                       jb->flags + c0, jb->resid + c0, jb->lengths + 2 * i))
        *jb->failed = 1;
      for (int w = 0; w < nw; ++w)
        for (int j = 0; j < d; ++j) jb->q_out[j * jb->ld + c0 + w] = Q[w * d + j];
      free(Q);
    } else if (jb->mode == 3) {
      double qt[OR_MAXJ], eps[OR_EXT_MAXN], qp[OR_MAXJ];
      for (int j = 0; j < d; ++j) qt[j] = jb->q_t[j * jb->ld + i];
      for (int k = 0; k < jb->ep->n; ++k) eps[k] = jb->eps[k * jb->ld_eps + i];
      int np = 0, w = -1;
      int st = extend_one(jb->rb, jb->cons, jb->nc, jb->p, jb->ep, jb->n_obs, jb->obs, jb->n_box, jb->box, q, qt,
                          eps, qp, &np, &w);
      for (int j = 0; j < d; ++j) jb->q_out[j * jb->ld + i] = qp[j];
      jb->flags[i] = (uint8_t)st;
      jb->n_points[i] = np;
      jb->winner[i] = w;
    } else {
      for (int j = 0; j < d; ++j) g[j] = jb->g[j * jb->ld + i];
      int ok = vjp_one(jb->rb, jb->cons, jb->nc, q, g, v);
      for (int j = 0; j < d; ++j) jb->v[j * jb->ld + i] = v[j];
      if (jb->flags) jb->flags[i] = (uint8_t)(ok ? 0 : OR_NONFINITE);
    }
  }
  return NULL;
}

static void run_jobs(or_job proto, int64_t n, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (n < nthreads) nthreads = n > 0 ? (int)n : 1;
  pthread_t th[256];
  or_job jobs[256];
  int64_t chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = proto;
    jobs[t].i0 = t * chunk;
    jobs[t].i1 = (t + 1) * chunk < n ? (t + 1) * chunk : n;
    if (jobs[t].i0 > n) jobs[t].i0 = n;
  }
  if (nthreads == 1) {
    job_run(&jobs[0]);
    return;
  }
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, job_run, &jobs[t]);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* Project n configurations (SoA, leading dimension ld). */
void or_project(const or_robot *rb, const or_constraint *cons, int nc, const or_params *p, int64_t n, int64_t ld,
                const double *q_in, double *q_out, uint8_t *flags, int32_t *iters, double *resid, int nthreads) {
  or_job jb;
  memset(&jb, 0, sizeof(jb));
  jb.rb = rb; jb.cons = cons; jb.nc = nc; jb.p = p; jb.ld = ld;
  jb.q_in = q_in; jb.q_out = q_out; jb.flags = flags; jb.iters = iters; jb.resid = resid;
  jb.mode = 0;
  run_jobs(jb, n, nthreads);
}

/* Collision verdict (1 = collides) and contact margin per configuration. */
void or_check(const or_robot *rb, int n_obs, const double *obs, int n_box, const double *box, int64_t n,
              int64_t ld, const double *q, uint8_t *hit, double *margin, int nthreads) {
  or_job jb;
  memset(&jb, 0, sizeof(jb));
  jb.rb = rb; jb.ld = ld; jb.q_in = q; jb.n_obs = n_obs; jb.obs = obs; jb.n_box = n_box; jb.box = box;
  jb.hit = hit; jb.margin = margin; jb.mode = 1;
  run_jobs(jb, n, nthreads);
}

/* VJP v = g - J^T (J J^T)^{-1} J g per configuration. */
void or_vjp(const or_robot *rb, const or_constraint *cons, int nc, int64_t n, int64_t ld, const double *q,
            const double *g, double *v, uint8_t *flags, int nthreads) {
  or_job jb;
  memset(&jb, 0, sizeof(jb));
  jb.rb = rb; jb.cons = cons; jb.nc = nc; jb.ld = ld; jb.q_in = q; jb.g = g; jb.v = v; jb.flags = flags;
  jb.mode = 2;
  run_jobs(jb, n, nthreads);
}

/* ParallelConstrainedExtend of n_ext extensions (SoA): q_s, q_t [d * ld],
 * eps [n * ld_eps] (particle offsets along the extension direction);
 * outputs q_proj [d * ld], status [n_ext], n_points, winner. */
void or_extend(const or_robot *rb, const or_constraint *cons, int nc, const or_params *p, const or_ext_params *ep,
               int n_obs, const double *obs, int n_box, const double *box, int64_t n_ext, int64_t ld,
               const double *q_s, const double *q_t, const double *eps, int64_t ld_eps, double *q_proj,
               uint8_t *status, int32_t *n_points, int32_t *winner, int nthreads) {
  or_job jb;
  memset(&jb, 0, sizeof(jb));
  jb.rb = rb; jb.cons = cons; jb.nc = nc; jb.p = p; jb.ld = ld; jb.ep = ep;
  jb.n_obs = n_obs; jb.obs = obs; jb.n_box = n_box; jb.box = box;
  jb.q_in = q_s; jb.q_t = q_t; jb.eps = eps; jb.ld_eps = ld_eps; jb.q_out = q_proj; jb.flags = status;
  jb.n_points = n_points; jb.winner = winner; jb.mode = 3;
  run_jobs(jb, n_ext, nthreads);
}

/* Path length and its gradient for n_paths paths of n_way waypoints (SoA
 * [d * ld], path p in columns p * n_way ..): L [n_paths], G [d * ld]. */
void or_path_length_grad(int d, int64_t n_paths, int n_way, int64_t ld, const double *Q, double *L, double *G) {
  double *B = (double *)malloc(sizeof(double) * (size_t)n_way * d * 2);
  if (!B) return;
  double *P = B, *Gp = B + (size_t)n_way * d;
  for (int64_t p = 0; p < n_paths; ++p) {
    for (int w = 0; w < n_way; ++w)
      for (int j = 0; j < d; ++j) P[w * d + j] = Q[j * ld + p * n_way + w];
    L[p] = path_length(d, n_way, P);
    if (G) {
      path_gradient(d, n_way, P, Gp);
      for (int w = 0; w < n_way; ++w)
        for (int j = 0; j < d; ++j) G[j * ld + p * n_way + w] = Gp[w * d + j];
    }
  }
  free(B);
}

/* Gradient path shortening of n_paths paths (SoA [d * ld], path p in columns
 * p * n_way ..): Q_out receives the final projected waypoints, flags / resid
 * their final projection, lengths [n_paths][2] the length before and after.
 * Returns 0 on success, 1 if scratch memory could not be allocated. */
int or_shorten(const or_robot *rb, const or_constraint *cons, int nc, const or_params *p, int64_t n_paths,
               int n_way, int64_t ld, const double *Q_in, int steps, double eta, double max_step, double *Q_out,
               uint8_t *flags, double *resid, double *lengths, int nthreads) {
  or_job jb;
  int failed = 0;
  memset(&jb, 0, sizeof(jb));
  jb.rb = rb; jb.cons = cons; jb.nc = nc; jb.p = p; jb.ld = ld; jb.q_in = Q_in; jb.q_out = Q_out;
  jb.flags = flags; jb.resid = resid; jb.n_way = n_way; jb.steps = steps; jb.eta = eta; jb.max_step = max_step;
  jb.lengths = lengths; jb.failed = &failed; jb.mode = 4;
  run_jobs(jb, n_paths, nthreads);
  return failed;
}
