// Kernel templates of the projection path, instantiated per problem class in
// inst_*.cu.  Building blocks are in mcp_device.cuh.
//
// Projection follows ParallelProject / getDescentStep of Algorithm 2 with the
// stacked constraint (Sec. IV-C) and the inner LM form
//     q <- q - J^T (J J^T + lambda I)^{-1} F(q)
// (Sec. IV-A, "Vectorized Levenberg-Marquardt"), stopping per configuration
// when ||F|| < tol, at the iteration cap, or on a step longer than MaxDistance.
#pragma once

#include <cfloat>

#include <math_constants.h>

#include "mcp_device.cuh"
#include "mcp_internal.h"
#include "mcp_problems.cuh"

namespace mcp {

constexpr unsigned FULL = 0xffffffffu;
// internal flag bits (never written out)
constexpr uint32_t FL_INT_FP32CONV = 1u << 8;   // FP32 residual passed; FP64 check pending
constexpr uint32_t FL_INT_NEEDS_F64 = 1u << 9;  // FP32 pivot below threshold: continue in FP64
constexpr uint32_t FL_INT_FORCE = 1u << 10;     // FP64 acceptance failed: one FP32 step before the next test

// Forms of getDescentStep (Alg. 2): the stacked inner step J^T (J J^T + lambda I)^-1 F,
// one inner step per constraint in turn (cyclic), or the stacked outer step
// (J^T J + lambda I)^-1 J^T F (a d x d system).
enum : int { FORM_STACKED = 0, FORM_CYCLIC = 1, FORM_OUTER = 2 };

// ---------------------------------------------------------------------------
// Stacked residual F(q) and Jacobian J(q)
// ---------------------------------------------------------------------------
template <class P, typename T>
struct Eval {
  V3<T> x[P::NC];    // POSE, PBND: world origin of T_a Q^-1; REL: p_b
  T G[P::NC][9];     // world -> error-frame rotation (POSE: P^-1_R; REL: P^-1_R R_a^T)
  V3<T> phi[P::NC];  // log of the error rotation
  T beta[P::NC];     // Jl^-1 coefficient
  V3<T> za[P::NC];   // AXIS: frame z axis; DIST: unit vector from x_a to x_b
  bool act[P::NC][6];  // PBND: component outside its bounds
  int hmode[P::NC];    // HULL: 0 inside, 1 nearest point on an edge, 2 at a vertex
  T hn[P::NC][2];      // HULL: outward normal of that edge
  T inv_norm;        // SPHERE: 1 / |q|
  V3<T> C[P::D];     // COM: mass-weighted CoM sum over the subtree of joint j
};

template <class P, class Ops, typename T, bool WANT_J>
__device__ __forceinline__ void residual(const ModelT<T> &m, const T (&q)[P::D], const Kin<P, T> &k,
                                         T (&F)[kdim<P>()], Eval<P, T> &e) {
  static_for<P::NC>([&](auto CC) {
    constexpr int c = decltype(CC)::value;
    constexpr int kind = P::ckind(c);
    constexpr int r0 = roff<P>(c);
    constexpr int cm = c + CBase<P>::value;  // model slot
    if constexpr (kind == K_SPHERE) {
      // F = |q| - r (configuration space)
      T n2 = T(0);
#pragma unroll
      for (int j = 0; j < P::D; ++j) n2 = fma_(q[j], q[j], n2);
      T inv = Ops::rsqrt_(n2);
      e.inv_norm = inv;
      F[r0] = n2 * inv - m.ctgt[cm][0];
    } else if constexpr (kind == K_AXIS) {
      // frame z axis parallel to world z: F = (z.x, z.y)
      constexpr int a = P::cfa(c);
      V3<T> za = col(k.fR[a], 2);
      e.za[c] = za;
      F[r0] = za.x;
      F[r0 + 1] = za.y;
    } else if constexpr (kind == K_POSE || kind == K_REL || kind == K_PBND) {
      T Pr[9];
      load_R(m.cPinv[cm], Pr);
      const V3<T> Pp = load_p(m.cPinv[cm]);
      T Rerr[9];
      V3<T> t;
      if constexpr (kind == K_POSE || kind == K_PBND) {
        // Eq. 1: T_err = (T_w^0)^-1 T_a (T_e^w)^-1
        constexpr int a = P::cfa(c);
        T Qr[9], RaQ[9];
        load_R(m.cQinv[cm], Qr);
        mul33(k.fR[a], Qr, RaQ);
        const V3<T> x = add_rot_t<7>(k.fp[a], k.fR[a], load_p(m.cQinv[cm]));
        mul33(Pr, RaQ, Rerr);
        const V3<T> tx = mulv(Pr, x);
        t = {tx.x + Pp.x, tx.y + Pp.y, tx.z + Pp.z};
        if constexpr (WANT_J) {
          e.x[c] = x;
#pragma unroll
          for (int i = 0; i < 9; ++i) e.G[c][i] = Pr[i];
        }
      } else {
        // Eq. 2: T_err = T_ref^-1 (T_a^-1 T_b); G = R_ref^T R_a^T
        constexpr int a = P::cfa(c), b = P::cfb(c);
        T G[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc)
            G[r * 3 + cc] = fma_(Pr[r * 3], k.fR[a][cc * 3],
                                 fma_(Pr[r * 3 + 1], k.fR[a][cc * 3 + 1], Pr[r * 3 + 2] * k.fR[a][cc * 3 + 2]));
        mul33(G, k.fR[b], Rerr);
        const V3<T> tx = mulv(G, sub(k.fp[b], k.fp[a]));
        t = {tx.x + Pp.x, tx.y + Pp.y, tx.z + Pp.z};
        if constexpr (WANT_J) {
          e.x[c] = k.fp[b];
#pragma unroll
          for (int i = 0; i < 9; ++i) e.G[c][i] = G[i];
        }
      }
      const auto lg = so3_log<Ops, T>(Rerr);
      if constexpr (WANT_J) {
        e.phi[c] = lg.phi;
        e.beta[c] = jl_inv_beta<T>(lg.theta, lg.s, lg.c);
      }
      F[r0] = t.x;
      F[r0 + 1] = t.y;
      F[r0 + 2] = t.z;
      F[r0 + 3] = lg.phi.x;
      F[r0 + 4] = lg.phi.y;
      F[r0 + 5] = lg.phi.z;
      if constexpr (kind == K_PBND) {
        // Eq. 1 with bounds B^w: each component's distance outside [lo, hi];
        // inside, the residual and its row of J are zero
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          const T lo = m.cB[cm][i], hi = m.cB[cm][6 + i], v = F[r0 + i];
          const bool below = v < lo, above = v > hi;
          F[r0 + i] = below ? v - lo : (above ? v - hi : T(0));
          if constexpr (WANT_J) e.act[c][i] = below || above;
        }
      }
    } else if constexpr (kind == K_PLANE || kind == K_LINE) {
      // origin of frame a in the task frame P: PLANE F = z, LINE F = (x, y)
      constexpr int a = P::cfa(c);
      const T *Pi = m.cPinv[cm];
      const V3<T> x = k.fp[a];
      if constexpr (kind == K_PLANE) {
        F[r0] = fma_(Pi[8], x.x, fma_(Pi[9], x.y, fma_(Pi[10], x.z, Pi[11])));
      } else {
        F[r0] = fma_(Pi[0], x.x, fma_(Pi[1], x.y, fma_(Pi[2], x.z, Pi[3])));
        F[r0 + 1] = fma_(Pi[4], x.x, fma_(Pi[5], x.y, fma_(Pi[6], x.z, Pi[7])));
      }
    } else if constexpr (kind == K_DIST) {
      // closed linkage: F = |x_b - x_a| - L
      constexpr int a = P::cfa(c), b = P::cfb(c);
      const V3<T> dv = sub(k.fp[b], k.fp[a]);
      const T n2 = fma_(dv.x, dv.x, fma_(dv.y, dv.y, dv.z * dv.z));
      const T inv = Ops::rsqrt_(n2);
      F[r0] = n2 * inv - m.ctgt[cm][0];
      if constexpr (WANT_J) e.za[c] = V3<T>{dv.x * inv, dv.y * inv, dv.z * inv};
    } else if constexpr (kind == K_COM || kind == K_HULL) {
      // Sec. V-C: x_com = sum_i m_i c_i / M with c_i = T_i com_i (the sum is
      // accumulated during FK).  With WANT_J the subtree sums C_j = m_j c_j +
      // sum over children are built in reverse topological order.
      if constexpr (WANT_J) {
        static_for<P::D>([&](auto JJ) {
          constexpr int j = P::D - 1 - decltype(JJ)::value;
          const V3<T> ci = add_rot_t<7>(k.p[j], k.R[j], V3<T>{m.com[j][0], m.com[j][1], m.com[j][2]});
          V3<T> acc{m.mass[j] * ci.x, m.mass[j] * ci.y, m.mass[j] * ci.z};
          static_for<P::D>([&](auto II) {
            constexpr int i = decltype(II)::value;
            if constexpr (i > j && P::parent(i) == j) acc = {acc.x + e.C[i].x, acc.y + e.C[i].y, acc.z + e.C[i].z};
          });
          e.C[j] = acc;
        });
      }
      if constexpr (kind == K_COM) {
        F[r0] = fma_(k.mc.x, m.inv_mass, -m.ctgt[cm][0]);
        F[r0 + 1] = fma_(k.mc.y, m.inv_mass, -m.ctgt[cm][1]);
      } else {
        // distance to the support polygon: F = c - nearest point (zero inside)
        const T cx = k.mc.x * m.inv_mass, cy = k.mc.y * m.inv_mass;
        T px, py, nx, ny;
        const int mode = polygon_nearest<T>(m.cB[cm], static_cast<int>(m.ctgt[cm][0]), cx, cy, px, py, nx, ny);
        F[r0] = cx - px;
        F[r0 + 1] = cy - py;
        if constexpr (WANT_J) {
          e.hmode[c] = mode;
          e.hn[c][0] = nx;
          e.hn[c][1] = ny;
        }
      }
    }
  });
}

// Jacobian of the stacked residual (world-frame geometric Jacobian rotated
// into each error frame).  Only entries where jnz() holds are written / read.
template <class P, typename T>
__device__ __forceinline__ void jacobian(const ModelT<T> &m, const T (&q)[P::D], const Kin<P, T> &k,
                                         const Eval<P, T> &e, T (&J)[kdim<P>()][P::D]) {
  static_for<P::NC>([&](auto CC) {
    constexpr int c = decltype(CC)::value;
    constexpr int kind = P::ckind(c);
    constexpr int r0 = roff<P>(c);
    constexpr int cm = c + CBase<P>::value;
    static_for<P::D>([&](auto JJ) {
      constexpr int j = decltype(JJ)::value;
      constexpr int s = col_sign<P>(c, j);
      constexpr bool rev = P::jtype(j) == REV;
      if constexpr (s != 0) {
        if constexpr (kind == K_SPHERE) {
          J[r0][j] = q[j] * e.inv_norm;
        } else if constexpr (kind == K_AXIS) {
          if constexpr (rev) {
            const V3<T> d = cross(k.z[j], e.za[c]);
            J[r0][j] = d.x;
            J[r0 + 1][j] = d.y;
          }
        } else if constexpr (kind == K_POSE || kind == K_REL || kind == K_PBND) {
          // translation rows: G (velocity of the error point); rotation rows: Jl^-1 G z_j.
          // REL: s = +1 for joints above b only, -1 above a only (Eq. 2, T_a^-1 T_b).
          // PBND: rows of components inside their bounds are zero.
          const V3<T> v = rev ? cross(k.z[j], sub(e.x[c], k.p[j])) : k.z[j];
          const V3<T> vt = mulv(e.G[c], v);
          T row[6] = {s > 0 ? vt.x : -vt.x, s > 0 ? vt.y : -vt.y, s > 0 ? vt.z : -vt.z, T(0), T(0), T(0)};
          if constexpr (rev) {
            const V3<T> w = jl_inv_apply(e.phi[c], e.beta[c], mulv(e.G[c], k.z[j]));
            row[3] = s > 0 ? w.x : -w.x;
            row[4] = s > 0 ? w.y : -w.y;
            row[5] = s > 0 ? w.z : -w.z;
          }
#pragma unroll
          for (int i = 0; i < (rev ? 6 : 3); ++i) {
            if constexpr (kind == K_PBND) J[r0 + i][j] = e.act[c][i] ? row[i] : T(0);
            else J[r0 + i][j] = row[i];
          }
        } else if constexpr (kind == K_PLANE || kind == K_LINE) {
          // rows of P^-1_R applied to the velocity of frame a's origin
          constexpr int a = P::cfa(c);
          const V3<T> v = rev ? cross(k.z[j], sub(k.fp[a], k.p[j])) : k.z[j];
          const T *Pi = m.cPinv[cm];
          if constexpr (kind == K_PLANE) {
            J[r0][j] = fma_(Pi[8], v.x, fma_(Pi[9], v.y, Pi[10] * v.z));
          } else {
            J[r0][j] = fma_(Pi[0], v.x, fma_(Pi[1], v.y, Pi[2] * v.z));
            J[r0 + 1][j] = fma_(Pi[4], v.x, fma_(Pi[5], v.y, Pi[6] * v.z));
          }
        } else if constexpr (kind == K_DIST) {
          // u . (velocity of x_b) for joints above b only, -u . (velocity of x_a) above a only
          constexpr int f = s > 0 ? P::cfb(c) : P::cfa(c);
          const V3<T> v = rev ? cross(k.z[j], sub(k.fp[f], k.p[j])) : k.z[j];
          const T d = fma_(e.za[c].x, v.x, fma_(e.za[c].y, v.y, e.za[c].z * v.z));
          J[r0][j] = s > 0 ? d : -d;
        } else if constexpr (kind == K_COM || kind == K_HULL) {
          // d x_com / d q_j = (1/M) z_j x (C_j - M_j o_j) (revolute), (M_j / M) z_j (prismatic)
          T g0, g1;
          if constexpr (rev) {
            const T Mj = m.msub[j];
            const V3<T> r{fma_(-Mj, k.p[j].x, e.C[j].x), fma_(-Mj, k.p[j].y, e.C[j].y), fma_(-Mj, k.p[j].z, e.C[j].z)};
            const V3<T> d = cross(k.z[j], r);
            g0 = d.x * m.inv_mass;
            g1 = d.y * m.inv_mass;
          } else {
            const T f = m.msub[j] * m.inv_mass;
            g0 = f * k.z[j].x;
            g1 = f * k.z[j].y;
          }
          if constexpr (kind == K_HULL) {  // inside: 0; on an edge: n n^T g; at a vertex: g
            if (e.hmode[c] == 0) {
              g0 = g1 = T(0);
            } else if (e.hmode[c] == 1) {
              const T sdot = fma_(e.hn[c][0], g0, e.hn[c][1] * g1);
              g0 = e.hn[c][0] * sdot;
              g1 = e.hn[c][1] * sdot;
            }
          }
          J[r0][j] = g0;
          J[r0 + 1][j] = g1;
        }
      }
    });
  });
}

// A = J J^T + lambda I (lower triangle), skipping structural zeros.
template <class P, typename T>
__device__ __forceinline__ void gram(const T (&J)[kdim<P>()][P::D], T lambda, T (&A)[kdim<P>() * (kdim<P>() + 1) / 2]) {
  constexpr int K = kdim<P>();
  static_for<K>([&](auto AA) {
    constexpr int a = decltype(AA)::value;
    static_for<a + 1>([&](auto BB) {
      constexpr int b = decltype(BB)::value;
      T s = (a == b) ? lambda : T(0);
      static_for<P::D>([&](auto JJ) {
        constexpr int j = decltype(JJ)::value;
        if constexpr (jnz<P>(a, j) && jnz<P>(b, j)) s = fma_(J[a][j], J[b][j], s);
      });
      A[tri(a, b)] = s;
    });
  });
}

// dq = J^T y
template <class P, typename T>
__device__ __forceinline__ void jt_mul(const T (&J)[kdim<P>()][P::D], const T (&y)[kdim<P>()], T (&dq)[P::D]) {
  static_for<P::D>([&](auto JJ) {
    constexpr int j = decltype(JJ)::value;
    T s = T(0);
    static_for<kdim<P>()>([&](auto AA) {
      constexpr int a = decltype(AA)::value;
      if constexpr (jnz<P>(a, j)) s = fma_(J[a][j], y[a], s);
    });
    dq[j] = s;
  });
}

// u = J g
template <class P, typename T>
__device__ __forceinline__ void j_mul(const T (&J)[kdim<P>()][P::D], const T (&g)[P::D], T (&u)[kdim<P>()]) {
  static_for<kdim<P>()>([&](auto AA) {
    constexpr int a = decltype(AA)::value;
    T s = T(0);
    static_for<P::D>([&](auto JJ) {
      constexpr int j = decltype(JJ)::value;
      if constexpr (jnz<P>(a, j)) s = fma_(J[a][j], g[j], s);
    });
    u[a] = s;
  });
}

// A = J^T J + lambda I (lower triangle of the d x d matrix), structural zeros skipped.
template <class P, typename T>
__device__ __forceinline__ void gram_outer(const T (&J)[kdim<P>()][P::D], T lambda, T (&A)[P::D * (P::D + 1) / 2]) {
  static_for<P::D>([&](auto II) {
    constexpr int i = decltype(II)::value;
    static_for<i + 1>([&](auto JJ) {
      constexpr int j = decltype(JJ)::value;
      T s = (i == j) ? lambda : T(0);
      static_for<kdim<P>()>([&](auto AA) {
        constexpr int a = decltype(AA)::value;
        if constexpr (jnz<P>(a, i) && jnz<P>(a, j)) s = fma_(J[a][i], J[a][j], s);
      });
      A[tri(i, j)] = s;
    });
  });
}

// ---------------------------------------------------------------------------
// Work items: a plain batch, or points on uneven segments.
// ---------------------------------------------------------------------------
template <typename T>
struct BatchSrc {
  const T *q;
  long long ld;
  __device__ __forceinline__ long long clamp_total(long long t) const { return t; }
  template <int D>
  __device__ __forceinline__ void load(long long item, T (&out)[D]) const {
    const bool ok = MCP_CHK(item, ld);
#pragma unroll
    for (int j = 0; j < D; ++j) out[j] = ok ? q[j * ld + item] : T(0);
  }
  // joints j0 .. j0 + N - 1 only
  template <int N>
  __device__ __forceinline__ void load_part(long long item, int j0, T (&out)[N]) const {
    const bool ok = MCP_CHK(item, ld);
#pragma unroll
    for (int j = 0; j < N; ++j) out[j] = ok ? q[(j0 + j) * ld + item] : T(0);
  }
};

template <typename T>
struct SegSrc {
  const T *start;
  const T *delta;
  long long ld;
  const long long *off;  // [n + 1]
  int n;
  // never hand out points past the end of the last segment
  __device__ __forceinline__ long long clamp_total(long long t) const {
    const long long dev_total = __ldg(&off[n]);
    return t < dev_total ? t : dev_total;
  }
  // last segment s with off[s] <= item (segments of length 0 are skipped)
  __device__ __forceinline__ int segment_of(long long item) const {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&off[mid]) <= item) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  }
  template <int D>
  __device__ __forceinline__ void load(long long item, T (&out)[D]) const {
    load_part<D>(item, 0, out);
  }
  // joints j0 .. j0 + N - 1 of the point
  template <int N>
  __device__ __forceinline__ void load_part(long long item, int j0, T (&out)[N]) const {
    const int s = segment_of(item);
    // the segment holds the item, and its start / delta columns exist
    const bool ok = MCP_CHK(s, n) && MCP_CHK(s, ld) && MCP_CHK(item - __ldg(&off[s]), __ldg(&off[s + 1]) - __ldg(&off[s]));
    if (!ok) {
#pragma unroll
      for (int j = 0; j < N; ++j) out[j] = T(0);
      return;
    }
    const T t = static_cast<T>(item - __ldg(&off[s]));
#pragma unroll
    for (int j = 0; j < N; ++j) out[j] = fma_(t, delta[(j0 + j) * ld + s], start[(j0 + j) * ld + s]);
  }
};

template <class P, class Src>
struct ProjArgs {
  ModelT<float> m;
  const ModelT<double> *__restrict__ m64;
  const double2 *__restrict__ tab;
  Src src;
  float *q_out;
  long long ld_out;
  uint8_t *flags;
  uint8_t *iters;
  double *resid;
  unsigned long long *counter;
  long long total;
  int chunk;
  int cap;
  float tol2;
  float lambda;
  float max_step2;
  float pivot;
  double tol2_64;
  double lambda64;
  float alpha;  // step scale of getDescentStep
  // fused collision check of every output (CHK kernels only)
  const CheckData *chk;
  const float *obs;
  const float *box;
  int n_obs;
  int n_box;
  uint8_t *hit;
  uint32_t *pairs;
};

// One step of iterative refinement of the LM solve with the residual formed
// from J itself (the corrected semi-normal equations of Bjorck):
//   r = F - J (J^T y) - lambda y,  y <- y + (L L^T)^{-1} r,  dq = J^T y.
// The Cholesky factor of J J^T + lambda I squares the condition number of J;
// in FP32 that alone moves a few percent of the 20-equation projections by
// more than 1e-4 rad from the exact-arithmetic iteration.  One refinement
// with the unsquared residual restores an error of order cond(J) eps.
template <class P, typename T>
__device__ __forceinline__ void refine_step(const T (&J)[kdim<P>()][P::D], const T (&F)[kdim<P>()], T lambda,
                                            const T (&L)[kdim<P>() * (kdim<P>() + 1) / 2], const T (&inv)[kdim<P>()],
                                            T (&y)[kdim<P>()], T (&dq)[P::D]) {
  constexpr int K = kdim<P>();
  T r[K];
  j_mul<P>(J, dq, r);
#pragma unroll
  for (int i = 0; i < K; ++i) r[i] = fma_(-lambda, y[i], F[i] - r[i]);
  cholesky_subst<K>(L, inv, r);
#pragma unroll
  for (int i = 0; i < K; ++i) y[i] += r[i];
  jt_mul<P>(J, y, dq);
}

// ---------------------------------------------------------------------------
// FP32 iteration (one pass of the ParallelProject loop for one configuration).
// Returns true when the configuration leaves the FP32 loop.
// ---------------------------------------------------------------------------
template <class P, class A, bool OUTER = false>
__device__ __forceinline__ bool newton_iter_f32(const A &a, float (&q)[P::D], int &it, uint32_t &fl) {
  constexpr int D = P::D, K = kdim<P>();
  const OpsF32 ops{a.tab};
  Kin<P, float> k;
  if constexpr (needs_fk<P>()) fk<P, needs_pos<P>()>(ops, a.m, q, k);
  float F[K];
  Eval<P, float> e;
  residual<P, OpsF32, float, true>(a.m, q, k, F, e);
  float r2 = 0.f;
#pragma unroll
  for (int i = 0; i < K; ++i) r2 = fmaf(F[i], F[i], r2);
  if (!(r2 <= FLT_MAX)) {
    fl |= FL_NONFINITE;
    return true;
  }
  if (r2 < a.tol2 && !(fl & FL_INT_FORCE)) {
    fl |= FL_INT_FP32CONV;
    return true;
  }
  if (it >= a.cap) {
    fl |= FL_CAP;
    return true;
  }
  float J[K][D];
  jacobian<P>(a.m, q, k, e, J);
  float dq[D];
  if constexpr (OUTER) {
    // (J^T J + lambda I) dq = J^T F, one refinement with r = J^T (F - J dq) - lambda dq
    float Am[D * (D + 1) / 2], inv[D];
    gram_outer<P>(J, a.lambda, Am);
    const float piv = cholesky_factor<D, OpsF32>(Am, inv);
    if (!(piv >= a.pivot)) {
      fl |= FL_INT_NEEDS_F64;
      return true;
    }
    jt_mul<P>(J, F, dq);
    cholesky_subst<D>(Am, inv, dq);
    float u[K], r[D];
    j_mul<P>(J, dq, u);
#pragma unroll
    for (int i = 0; i < K; ++i) u[i] = F[i] - u[i];
    jt_mul<P>(J, u, r);
#pragma unroll
    for (int j = 0; j < D; ++j) r[j] = fmaf(-a.lambda, dq[j], r[j]);
    cholesky_subst<D>(Am, inv, r);
#pragma unroll
    for (int j = 0; j < D; ++j) dq[j] += r[j];
  } else {
    float Am[K * (K + 1) / 2], inv[K];
    gram<P>(J, a.lambda, Am);
    const float piv = cholesky_factor<K, OpsF32>(Am, inv);
    if (!(piv >= a.pivot)) {  // also catches NaN: finish this configuration in FP64
      fl |= FL_INT_NEEDS_F64;
      return true;
    }
    float y[K];
#pragma unroll
    for (int i = 0; i < K; ++i) y[i] = F[i];
    cholesky_subst<K>(Am, inv, y);
    jt_mul<P>(J, y, dq);
    refine_step<P>(J, F, a.lambda, Am, inv, y, dq);
  }
  float s2 = 0.f;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    dq[j] *= a.alpha;
    s2 = fmaf(dq[j], dq[j], s2);
  }
  if (a.max_step2 > 0.f && s2 > a.max_step2) {
    fl |= FL_DIV;
    return true;
  }
#pragma unroll
  for (int j = 0; j < D; ++j) q[j] -= dq[j];
  ++it;
  fl &= ~FL_INT_FORCE;
  if (!(s2 <= FLT_MAX)) {
    fl |= FL_NONFINITE;
    return true;
  }
  return false;
}

// One FP32 LM step of the (sub-)problem S at q, applied in place: the unit of
// the cyclic form.  Returns false (q untouched) if a Cholesky pivot falls below
// the FP64 re-solve threshold.
template <class S, class A>
__device__ __forceinline__ bool substep_f32(const A &a, float (&q)[S::D]) {
  constexpr int D = S::D, K = kdim<S>();
  const OpsF32 ops{a.tab};
  Kin<S, float> k;
  if constexpr (needs_fk<S>()) fk<S, needs_pos<S>()>(ops, a.m, q, k);
  float F[K];
  Eval<S, float> e;
  residual<S, OpsF32, float, true>(a.m, q, k, F, e);
  float J[K][D];
  jacobian<S>(a.m, q, k, e, J);
  float Am[K * (K + 1) / 2], inv[K];
  gram<S>(J, a.lambda, Am);
  const float piv = cholesky_factor<K, OpsF32>(Am, inv);
  if (!(piv >= a.pivot)) return false;
  float y[K], dq[D];
#pragma unroll
  for (int i = 0; i < K; ++i) y[i] = F[i];
  cholesky_subst<K>(Am, inv, y);
  jt_mul<S>(J, y, dq);
  refine_step<S>(J, F, a.lambda, Am, inv, y, dq);
#pragma unroll
  for (int j = 0; j < D; ++j) q[j] -= a.alpha * dq[j];
  return true;
}

// One sweep of the cyclic getDescentStep (Sec. IV-C): the stopping test on the
// stacked F, then one LM step per constraint in stack order, each at the
// configuration the previous one produced.  MaxDistance applies to the whole
// sweep; a pivot below the threshold hands the sweep, from its start, to FP64.
template <class P, class A>
__device__ __forceinline__ bool cyclic_iter_f32(const A &a, float (&q)[P::D], int &it, uint32_t &fl) {
  constexpr int D = P::D, K = kdim<P>();
  {
    const OpsF32 ops{a.tab};
    Kin<P, float> k;
    if constexpr (needs_fk<P>()) fk<P, needs_pos<P>()>(ops, a.m, q, k);
    float F[K];
    Eval<P, float> e;
    residual<P, OpsF32, float, false>(a.m, q, k, F, e);
    float r2 = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) r2 = fmaf(F[i], F[i], r2);
    if (!(r2 <= FLT_MAX)) {
      fl |= FL_NONFINITE;
      return true;
    }
    if (r2 < a.tol2 && !(fl & FL_INT_FORCE)) {
      fl |= FL_INT_FP32CONV;
      return true;
    }
    if (it >= a.cap) {
      fl |= FL_CAP;
      return true;
    }
  }
  float q0[D];
#pragma unroll
  for (int j = 0; j < D; ++j) q0[j] = q[j];
  bool ok = true;
  static_for<P::NC>([&](auto CC) {
    if (ok) ok = substep_f32<Sub<P, decltype(CC)::value>>(a, q);
  });
  float s2 = 0.f;
#pragma unroll
  for (int j = 0; j < D; ++j) s2 = fmaf(q[j] - q0[j], q[j] - q0[j], s2);
  if (!ok || (a.max_step2 > 0.f && s2 > a.max_step2)) {
#pragma unroll
    for (int j = 0; j < D; ++j) q[j] = q0[j];
    fl |= ok ? FL_DIV : FL_INT_NEEDS_F64;
    return true;
  }
  ++it;
  fl &= ~FL_INT_FORCE;
  if (!(s2 <= FLT_MAX)) {
    fl |= FL_NONFINITE;
    return true;
  }
  return false;
}

// ---------------------------------------------------------------------------
// FP64 pieces used by the acceptance pass.
// ---------------------------------------------------------------------------
template <class P>
__host__ __device__ constexpr bool axis_only() {
  for (int c = 0; c < P::NC; ++c)
    if (P::ckind(c) != K_AXIS) return false;
  return true;
}
template <class P>
__host__ __device__ constexpr int chain_len(int link) {
  int n = 0;
  for (int l = link; l >= 0; l = P::parent(l)) ++n;
  return n;
}
template <class P>
__host__ __device__ constexpr int chain_at(int link, int k) {  // k-th joint from `link` towards the root
  int l = link;
  for (int i = 0; i < k; ++i) l = P::parent(l);
  return l;
}
// v <- R v for a fixed rotation given by its code (signed permutation: no arithmetic) or dense
template <int CODE>
__device__ __forceinline__ V3<double> xrot_apply(const double *X, V3<double> v) {
  if constexpr (CODE == XR_GENERIC) {
    return {fma(X[0], v.x, fma(X[1], v.y, X[2] * v.z)), fma(X[4], v.x, fma(X[5], v.y, X[6] * v.z)),
            fma(X[8], v.x, fma(X[9], v.y, X[10] * v.z))};
  } else {
    double o[3] = {0.0, 0.0, 0.0};
    const double in[3] = {v.x, v.y, v.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) o[xr_perm(CODE, k)] = xr_neg(CODE, k) ? -in[k] : in[k];
    return {o[0], o[1], o[2]};
  }
}

// Squared FP64 residual of axis-alignment constraints: only the frame's z axis
// enters F, so one vector is carried from the frame to the root,
//   z = X_0 Rz(q_0) ... X_l Rz(q_l) Xf e_z,
// at 4 FP64 operations per revolute joint (plus its sin/cos) instead of a
// full rotation product.  A revolute root joint whose axis is world z (X_0
// without rotation) turns z about world z, which leaves z.x^2 + z.y^2 = |F|^2
// unchanged: its rotation is skipped.
template <class P>
__host__ __device__ constexpr bool norm_invariant_root(int j) {
  return P::parent(j) < 0 && P::jtype(j) == REV && P::xrot(j) == XR_IDENTITY;
}
template <class P, class Ops, typename Q>
__device__ __forceinline__ double axis_residual2_f64(const Ops &ops, const ModelT<double> &m, const Q (&q)[P::D]) {
  double r2 = 0.0;
  static_for<P::NC>([&](auto CC) {
    constexpr int c = decltype(CC)::value;
    constexpr int f = P::cfa(c);
    constexpr int l = P::frame_link(f);
    V3<double> v = xrot_apply<P::frot(f)>(m.fX[f], V3<double>{0.0, 0.0, 1.0});
    static_for<chain_len<P>(l)>([&](auto KK) {
      constexpr int j = chain_at<P>(l, decltype(KK)::value);
      if constexpr (norm_invariant_root<P>(j)) {
        return;
      } else if constexpr (P::jtype(j) == REV) {
        double sn, cs;
        ops.sincos(q[j], sn, cs);
        v = {fma(cs, v.x, -(sn * v.y)), fma(sn, v.x, cs * v.y), v.z};
      }
      v = xrot_apply<P::xrot(j)>(m.X[j], v);
    });
    r2 = fma(v.x, v.x, fma(v.y, v.y, r2));
  });
  return r2;
}

template <class P, class Ops>
__device__ __forceinline__ double residual2_f64(const Ops &ops, const ModelT<double> &m,
                                                const double (&q)[P::D]) {
  if constexpr (axis_only<P>()) return axis_residual2_f64<P>(ops, m, q);
  constexpr int K = kdim<P>();
  Kin<P, double> k;
  if constexpr (needs_fk<P>()) fk<P, needs_pos<P>()>(ops, m, q, k);
  double F[K];
  Eval<P, double> e;
  residual<P, Ops, double, false>(m, q, k, F, e);
  double r2 = 0.0;
#pragma unroll
  for (int i = 0; i < K; ++i) r2 = fma(F[i], F[i], r2);
  return r2;
}

// The same for an FP32 configuration (the acceptance of an FP32 iterate): the
// axis form takes the FP32 angles straight into the split sin/cos.
template <class P, class Ops>
__device__ __forceinline__ double residual2_f64(const Ops &ops, const ModelT<double> &m, const float (&q)[P::D]) {
  if constexpr (axis_only<P>()) {
    return axis_residual2_f64<P>(ops, m, q);
  } else {
    double qd[P::D];
#pragma unroll
    for (int j = 0; j < P::D; ++j) qd[j] = static_cast<double>(q[j]);
    return residual2_f64<P>(ops, m, qd);
  }
}

// One LM step entirely in FP64 at q (the re-solve of a badly conditioned
// system).  J and the factorisation live in local memory (runtime-indexed
// loops) so that this rare path does not raise the register budget of the
// FP32 loop.  Returns false if the FP64 system is singular as well.
template <class P, bool OUTER = false>
__device__ __noinline__ bool lm_step_f64(const OpsF64Table ops, const ModelT<double> *__restrict__ m,
                                         const double *q_in, double lambda, double *dq_out) {
  constexpr int D = P::D, K = kdim<P>();
  double q[D];
#pragma unroll
  for (int j = 0; j < D; ++j) q[j] = q_in[j];
  Kin<P, double> k;
  if constexpr (needs_fk<P>()) fk<P, needs_pos<P>()>(ops, *m, q, k);
  double F[K];
  Eval<P, double> e;
  residual<P, OpsF64Table, double, true>(*m, q, k, F, e);
  double J[K][D];
#pragma unroll 1
  for (int a = 0; a < K; ++a)
#pragma unroll 1
    for (int j = 0; j < D; ++j) J[a][j] = 0.0;
  jacobian<P>(*m, q, k, e, J);
  if constexpr (OUTER) {
    // (J^T J + lambda I) dq = J^T F
    double L[D][D], b[D];
#pragma unroll 1
    for (int i = 0; i < D; ++i) {
      double t = 0.0;
#pragma unroll 1
      for (int a = 0; a < K; ++a) t = fma(J[a][i], F[a], t);
      b[i] = t;
#pragma unroll 1
      for (int j = 0; j <= i; ++j) {
        double s = (i == j) ? lambda : 0.0;
#pragma unroll 1
        for (int a = 0; a < K; ++a) s = fma(J[a][i], J[a][j], s);
        L[i][j] = s;
      }
    }
#pragma unroll 1
    for (int j = 0; j < D; ++j) {
      double s = L[j][j];
#pragma unroll 1
      for (int t = 0; t < j; ++t) s = fma(-L[j][t], L[j][t], s);
      if (!(s > 0.0)) return false;
      L[j][j] = sqrt(s);
#pragma unroll 1
      for (int i = j + 1; i < D; ++i) {
        double t2 = L[i][j];
#pragma unroll 1
        for (int t = 0; t < j; ++t) t2 = fma(-L[i][t], L[j][t], t2);
        L[i][j] = t2 / L[j][j];
      }
    }
#pragma unroll 1
    for (int i = 0; i < D; ++i) {
      double t = b[i];
#pragma unroll 1
      for (int u = 0; u < i; ++u) t = fma(-L[i][u], b[u], t);
      b[i] = t / L[i][i];
    }
#pragma unroll 1
    for (int i = D - 1; i >= 0; --i) {
      double t = b[i];
#pragma unroll 1
      for (int u = i + 1; u < D; ++u) t = fma(-L[u][i], b[u], t);
      b[i] = t / L[i][i];
    }
#pragma unroll 1
    for (int j = 0; j < D; ++j) dq_out[j] = b[j];
    return true;
  } else {
  double L[K][K];
#pragma unroll 1
  for (int a = 0; a < K; ++a) {
#pragma unroll 1
    for (int b = 0; b <= a; ++b) {
      double s = (a == b) ? lambda : 0.0;
#pragma unroll 1
      for (int j = 0; j < D; ++j) s = fma(J[a][j], J[b][j], s);
      L[a][b] = s;
    }
  }
#pragma unroll 1
  for (int j = 0; j < K; ++j) {
    double s = L[j][j];
#pragma unroll 1
    for (int t = 0; t < j; ++t) s = fma(-L[j][t], L[j][t], s);
    if (!(s > 0.0)) return false;
    L[j][j] = sqrt(s);
#pragma unroll 1
    for (int i = j + 1; i < K; ++i) {
      double t2 = L[i][j];
#pragma unroll 1
      for (int t = 0; t < j; ++t) t2 = fma(-L[i][t], L[j][t], t2);
      L[i][j] = t2 / L[j][j];
    }
  }
  double y[K];
#pragma unroll 1
  for (int i = 0; i < K; ++i) {
    double s = F[i];
#pragma unroll 1
    for (int t = 0; t < i; ++t) s = fma(-L[i][t], y[t], s);
    y[i] = s / L[i][i];
  }
#pragma unroll 1
  for (int i = K - 1; i >= 0; --i) {
    double s = y[i];
#pragma unroll 1
    for (int t = i + 1; t < K; ++t) s = fma(-L[t][i], y[t], s);
    y[i] = s / L[i][i];
  }
#pragma unroll 1
  for (int j = 0; j < D; ++j) {
    double s = 0.0;
#pragma unroll 1
    for (int a = 0; a < K; ++a) s = fma(J[a][j], y[a], s);
    dq_out[j] = s;
  }
  return true;
  }
}

// Heron refinement of an FP32 square root: one Newton step in FP64 brings the
// FP32 estimate (relative error ~6e-8) to ~1e-14.
__device__ __forceinline__ double sqrt_refined(double v) {
  if (!(v > 0.0) || !(v <= DBL_MAX)) return sqrt(v);
  const float r0f = sqrtf(static_cast<float>(v));
  if (r0f == 0.0f) return sqrt(v);
  const double r0 = static_cast<double>(r0f);
  const double h = static_cast<double>(0.5f / r0f);
  return fma(fma(-r0, r0, v), h, r0);
}

// Remaining steps of one configuration in FP64 (rounded to the FP32 output):
// taken when the FP32 residual test passed but the FP64 one did not, or when
// the FP32 Cholesky pivot fell below the threshold.  Rare, so it lives out of
// line (its registers and local arrays stay off the FP32 loop).  Updates q,
// qd, it, fl; returns the final squared FP64 residual.
template <class P, int FORM, class A>
__device__ __noinline__ double finish_f64(const A &a, float *q, double *qd, int *it_io, uint32_t *fl_io, double r2,
                                          bool was_conv) {
  constexpr int D = P::D;
  constexpr bool CYC = FORM == FORM_CYCLIC;
  const double alpha = static_cast<double>(a.alpha);
  const OpsF64Table ops{a.tab};
  const ModelT<double> &m = *a.m64;
  int it = *it_io;
  uint32_t fl = *fl_io;
  bool conv = r2 < a.tol2_64;
  double qq[D];
#pragma unroll 1
  for (int j = 0; j < D; ++j) qq[j] = qd[j];
  while (!conv && it < a.cap) {
    fl |= FL_RESOLVE;
    if constexpr (CYC) {
      // one cyclic sweep in FP64 (each sub-step's result rounded to the FP32 output)
      float q0[D];
#pragma unroll 1
      for (int j = 0; j < D; ++j) q0[j] = q[j];
      bool sing = false;
      static_for<P::NC>([&](auto CC) {
        if (sing) return;
        double dq[D];
        if (!lm_step_f64<Sub<P, decltype(CC)::value>>(ops, a.m64, qq, a.lambda64, dq)) {
          sing = true;
          return;
        }
#pragma unroll 1
        for (int j = 0; j < D; ++j) {
          q[j] = static_cast<float>(qq[j] - alpha * dq[j]);
          qq[j] = static_cast<double>(q[j]);
        }
      });
      if (sing) {
        fl |= FL_NONFINITE;
        break;
      }
      double s2 = 0.0;
#pragma unroll 1
      for (int j = 0; j < D; ++j) {
        const double dj = qq[j] - static_cast<double>(q0[j]);
        s2 = fma(dj, dj, s2);
      }
      if (a.max_step2 > 0.f && s2 > static_cast<double>(a.max_step2)) {
#pragma unroll 1
        for (int j = 0; j < D; ++j) {
          q[j] = q0[j];
          qq[j] = static_cast<double>(q0[j]);
        }
        fl |= FL_DIV;
        break;
      }
    } else {
      double dq[D];
      if (!lm_step_f64<P, FORM == FORM_OUTER>(ops, a.m64, qq, a.lambda64, dq)) {
        fl |= FL_NONFINITE;
        break;
      }
      double s2 = 0.0;
#pragma unroll 1
      for (int j = 0; j < D; ++j) {
        dq[j] *= alpha;
        s2 = fma(dq[j], dq[j], s2);
      }
      if (a.max_step2 > 0.f && s2 > static_cast<double>(a.max_step2)) {
        fl |= FL_DIV;
        break;
      }
#pragma unroll 1
      for (int j = 0; j < D; ++j) {
        q[j] = static_cast<float>(qq[j] - dq[j]);
        qq[j] = static_cast<double>(q[j]);
      }
    }
    ++it;
    r2 = residual2_f64<P>(OpsF64Split{a.tab}, m, qq);  // qq holds FP32 values
    if (!(r2 <= DBL_MAX)) {
      fl |= FL_NONFINITE;
      break;
    }
    conv = r2 < a.tol2_64;
  }
  if (conv) fl |= FL_CONV;
  else if (!(fl & (FL_NONFINITE | FL_DIV))) fl |= FL_CAP | (was_conv ? FL_ACCEPT_FAIL : 0u);
#pragma unroll 1
  for (int j = 0; j < D; ++j) qd[j] = qq[j];
  *it_io = it;
  *fl_io = fl;
  return r2;
}

// Acceptance of one configuration that left the FP32 loop: the FP32 iterate
// is re-checked with the FP64 residual.  If the FP32 test was too optimistic
// and steps remain, the configuration goes back to the FP32 loop for one more
// step (retry allowed: returns true, nothing written); otherwise, or when the
// FP32 pivot was too small, finish_f64 takes the remaining steps in FP64.
// Writes q (if changed), flags, iters and resid.
template <class P, int FORM, class A>
__device__ __forceinline__ bool accept_one(const A &a, long long item, int it, uint32_t fl, bool retry_ok = false) {
  constexpr int D = P::D;
  const ModelT<double> &m = *a.m64;
  float q[D];
  const bool ok = MCP_CHK(item, a.ld_out);
#pragma unroll
  for (int j = 0; j < D; ++j) q[j] = ok ? a.q_out[j * a.ld_out + item] : 0.f;
  double r2 = residual2_f64<P>(OpsF64Split{a.tab}, m, q);
  if (retry_ok && (fl & FL_INT_FP32CONV) && !(r2 < a.tol2_64) && r2 <= DBL_MAX && it < a.cap) return true;
  if (fl & (FL_INT_FP32CONV | FL_INT_NEEDS_F64)) {
    const bool was_conv = (fl & FL_INT_FP32CONV) != 0;
    fl &= ~(FL_INT_FP32CONV | FL_INT_NEEDS_F64);
    if (r2 < a.tol2_64) {
      fl |= FL_CONV;
    } else {
      float qf[D];
      double qdd[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        qf[j] = q[j];
        qdd[j] = static_cast<double>(q[j]);
      }
      r2 = finish_f64<P, FORM>(a, qf, qdd, &it, &fl, r2, was_conv);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        if (ok) a.q_out[j * a.ld_out + item] = qf[j];
        q[j] = qf[j];
      }
    }
  }
  // limits in FP32: the FP32 copies of the bounds are rounded outwards
  // (lower up, upper down), so for an FP32 value q the FP32 comparison equals
  // the comparison with the FP64 bound
#pragma unroll
  for (int j = 0; j < D; ++j)
    if (q[j] < a.m.lower[j] || q[j] > a.m.upper[j]) fl |= FL_LIMITS;
  if (ok) {
    a.flags[item] = static_cast<uint8_t>(fl & 0xffu);
    a.iters[item] = static_cast<uint8_t>(it > 255 ? 255 : it);
    a.resid[item] = sqrt_refined(r2);
  }
  return false;
}

// ---------------------------------------------------------------------------
// Collision check (CollisionFree of Alg. 2): link spheres against obstacle
// spheres and boxes.  One thread per configuration.
//
// FP32 path: coordinates are shifted by the obstacle centroid o (applied to
// the robot base translations and to the staged obstacles), and the sphere
// test |c_s - c_o| < r_s + r_o is evaluated in the expanded form
//     c_s . (-2 c_o) + (|c_o|^2 - r_o^2) + r_s (-2 r_o)  <  -(|c_s|^2 - r_s^2)
// with the obstacle terms precomputed: 4 FMA + 1 min per pair.  Spheres are
// processed in register blocks of 8 per link (ILP), obstacles are read from
// shared memory with one broadcast load each; the configuration exits after
// the first block that overlaps an obstacle.  In the shifted frame |c| stays
// within a few metres, so the FP32 cancellation error of the expanded form
// stays below ~1e-5 m in distance (verified against the FP64 oracle).
// FP64 path: the plain difference form, one sphere at a time.
// ---------------------------------------------------------------------------
template <class P, typename T>
struct CheckArgs {
  ModelT<T> m;
  SphereTable<T> st;
  const T *obs;  // FP32: [n_obs * 8] (-2c, |c|^2 - r^2, -2r, pad) in the shifted frame; FP64: [n_obs * 4]
  const T *box;  // [n_box * 6] (FP32: shifted)
  int n_obs;
  int n_box;
  const T *q;
  long long ld;
  long long n;
  uint8_t *out;
  uint32_t *pairs;  // optional: number of sphere-obstacle pairs tested per configuration
  const double2 *tab;
};

template <typename T>
__device__ __forceinline__ T max_(T a, T b) {
  return a > b ? a : b;
}

template <typename T>
__device__ __forceinline__ bool box_hits(V3<T> c, T rs, const T *s_box, int n_box) {
  for (int b = 0; b < n_box; ++b) {
    const T *bx = s_box + 6 * b;
    const T ex = max_(max_(bx[0] - c.x, c.x - bx[3]), T(0));
    const T ey = max_(max_(bx[1] - c.y, c.y - bx[4]), T(0));
    const T ez = max_(max_(bx[2] - c.z, c.z - bx[5]), T(0));
    if (fma_(ex, ex, fma_(ey, ey, ez * ez)) < rs * rs) return true;
  }
  return false;
}

template <typename T>
__device__ __forceinline__ bool sphere_hits_plain(V3<T> c, T rs, const T *s_obs, int n_obs, const T *s_box, int n_box) {
  for (int o = 0; o < n_obs; ++o) {
    const T dx = c.x - s_obs[4 * o], dy = c.y - s_obs[4 * o + 1], dz = c.z - s_obs[4 * o + 2];
    const T rr = rs + s_obs[4 * o + 3];
    if (fma_(dx, dx, fma_(dy, dy, dz * dz)) < rr * rr) return true;
  }
  return box_hits<T>(c, rs, s_box, n_box);
}

constexpr int SPH_BLOCK = 8;

// A rotation by value (nine registers across a call).
struct Rot9 {
  float r[9];
};

// Obstacle records in shared memory, two obstacles per 48-byte pair so that
// the broad phase tests two obstacles per packed FP32x2 instruction:
//   A = (gx0, gx1, gy0, gy1), B = (gz0, gz1, gw0, gw1), C = (g20, g21, 0, 0)
// with g = -2 c, gw = |c|^2 - r^2, g2 = -2 r (the expanded overlap test
// below).  An odd count is padded with a record that never overlaps.
__host__ __device__ constexpr int obs_pairs(int n_obs) { return (n_obs + 1) / 2; }
// The records of the chunk spheres (one per OBS_CHUNK consecutive obstacles,
// same form) follow the obstacles' pairs, also in pairs: one chunk pair per
// 32 obstacles.
__host__ __device__ constexpr size_t obs_smem_bytes(int n_obs, int n_box) {
  return sizeof(float) * (12 * static_cast<size_t>(obs_pairs(n_obs)) + 12 * static_cast<size_t>(obs_pairs(obs_chunks(n_obs))) +
                          6 * static_cast<size_t>(n_box));
}
// Obstacle o's five values from its pair.
struct ObsRec {
  float gx, gy, gz, gw, g2;
};
__device__ __forceinline__ ObsRec obs_rec(const float4 *s_pair, int o) {
  const float *f = reinterpret_cast<const float *>(s_pair + 3 * (o >> 1));
  const int h = o & 1;
  return ObsRec{f[h], f[2 + h], f[4 + h], f[6 + h], f[8 + h]};
}

// Spheres [s0, e) of one link placed by (R, p), with the link's bounding
// sphere lb (local): the boxes the bound overlaps, then, per 32 obstacles, the bounding sphere
// against their two chunk spheres (CHUNKS, scenes of more than 32 obstacles)
// and the obstacles of the chunks it overlaps (broad phase, two records per
// FP32x2 instruction), then the
// link's spheres in blocks of 8 against the candidate obstacles (narrow
// phase, two spheres per instruction).  Every packed lane is an IEEE fma with
// round-to-nearest, so each test is bit-identical to the scalar chain
// fmaf(x, gx, fmaf(y, gy, fmaf(z, gz, fmaf(r, g2, gw)))).  One out-of-line
// copy serves every link of every kernel (inlined per link, the unrolled
// broad phase made kernels with many links instruction-cache bound).
template <bool CHUNKS>
static __device__ __noinline__ bool link_hits_f32(const Rot9 Rr, V3<float> p, int s0, int e, const float *lb,
                                                  const SphereTable<float> &st, const float4 *s_pair, int n_obs,
                                                  const float *s_box, int n_box, uint32_t *tests_io) {
  if (s0 >= e) return false;
  const float(&R)[9] = Rr.r;
  uint32_t tests = *tests_io;
  bool hit = false;
  const V3<float> bc = add_rot_t<7>(p, R, V3<float>{lb[0], lb[1], lb[2]});
  const float br = lb[3];
  // boxes: the link's spheres against a box only where the link's bounding
  // sphere (which contains them) overlaps it
  for (int b = 0; b < n_box && !hit; ++b) {
    const float *bx = s_box + 6 * b;
    if (!box_hits<float>(bc, br, bx, 1)) continue;
    for (int s = s0; s < e && !hit; ++s) {
      const V3<float> c = add_rot_t<7>(p, R, V3<float>{st.s[s][0], st.s[s][1], st.s[s][2]});
      if (box_hits<float>(c, st.s[s][3], bx, 1)) hit = true;
    }
  }
  const float kb = fmaf(bc.x, bc.x, fmaf(bc.y, bc.y, fmaf(bc.z, bc.z, -br * br)));
  const float2 bx2 = make_float2(bc.x, bc.x), by2 = make_float2(bc.y, bc.y), bz2 = make_float2(bc.z, bc.z),
               br2 = make_float2(br, br);
  const float4 *s_chunk = s_pair + 3 * obs_pairs(n_obs);
  // the bounding sphere's 4-FMA test against the records pr[pp] (two per pair)
  auto pair_bits = [&](const float4 *pr, int pp) -> unsigned {
    const float4 A = pr[3 * pp], B = pr[3 * pp + 1], C = pr[3 * pp + 2];
    float2 v = __ffma2_rn(br2, make_float2(C.x, C.y), make_float2(B.z, B.w));
    v = __ffma2_rn(bz2, make_float2(B.x, B.y), v);
    v = __ffma2_rn(by2, make_float2(A.z, A.w), v);
    v = __ffma2_rn(bx2, make_float2(A.x, A.y), v);
    return (v.x < -kb ? 1u : 0u) | (v.y < -kb ? 2u : 0u);
  };
  for (int o0 = 0; o0 < n_obs && !hit; o0 += 32) {
    const int cnt = min(32, n_obs - o0);
    const float4 *pr = s_pair + 3 * (o0 >> 1);
    unsigned cand = 0u;
    if (CHUNKS && n_obs > 32) {
      // the two chunks of these 32 obstacles first (a chunk's sphere contains
      // its obstacles, so an obstacle the bound overlaps lies in a chunk it
      // overlaps)
      const unsigned chunks = pair_bits(s_chunk, o0 >> 5);
      tests += cnt > OBS_CHUNK ? 2u : 1u;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!((chunks >> h) & 1u)) continue;
        const int c0 = h * OBS_CHUNK, cc = min(OBS_CHUNK, cnt - c0);
        if (cc <= 0) continue;
        if (cc == OBS_CHUNK) {  // full chunk: unrolled, compile-time bit positions
#pragma unroll
          for (int pp = 0; pp < OBS_CHUNK / 2; ++pp) cand |= pair_bits(pr, h * (OBS_CHUNK / 2) + pp) << (c0 + 2 * pp);
        } else {  // the padded record of an odd count never overlaps
          for (int pp = 0; pp < obs_pairs(cc); ++pp) cand |= pair_bits(pr, h * (OBS_CHUNK / 2) + pp) << (c0 + 2 * pp);
        }
        tests += static_cast<uint32_t>(cc);
      }
    } else {
      // 32 obstacles or fewer: the chunks span the whole scene and rarely
      // prune; every obstacle against the bound
      if (cnt == 32) {  // full chunk: unrolled, compile-time bit positions
#pragma unroll
        for (int pp = 0; pp < 16; ++pp) cand |= pair_bits(pr, pp) << (2 * pp);
      } else {  // the padded record of an odd count never overlaps
        for (int pp = 0; pp < obs_pairs(cnt); ++pp) cand |= pair_bits(pr, pp) << (2 * pp);
      }
      tests += static_cast<uint32_t>(cnt);
    }
    if (!cand) continue;
    for (int sb = s0; sb < e && !hit; sb += SPH_BLOCK) {
      const int count = min(SPH_BLOCK, e - sb);
      static_assert(SPH_BLOCK % 2 == 0, "spheres are tested in pairs");
      float2 cx[SPH_BLOCK / 2], cy[SPH_BLOCK / 2], cz[SPH_BLOCK / 2], rs[SPH_BLOCK / 2], ks[SPH_BLOCK / 2];
#pragma unroll
      for (int b = 0; b < SPH_BLOCK; ++b) {
        const int s = sb + (b < count ? b : 0);
        const V3<float> c = add_rot_t<7>(p, R, V3<float>{st.s[s][0], st.s[s][1], st.s[s][2]});
        const float r = st.s[s][3];
        const float k = (b < count) ? fmaf(c.x, c.x, fmaf(c.y, c.y, fmaf(c.z, c.z, -r * r))) : FLT_MAX;  // pad: never a hit
        float *dx = reinterpret_cast<float *>(&cx[b / 2]), *dy = reinterpret_cast<float *>(&cy[b / 2]),
              *dz = reinterpret_cast<float *>(&cz[b / 2]), *dr = reinterpret_cast<float *>(&rs[b / 2]),
              *dk = reinterpret_cast<float *>(&ks[b / 2]);
        dx[b & 1] = c.x;
        dy[b & 1] = c.y;
        dz[b & 1] = c.z;
        dr[b & 1] = r;
        dk[b & 1] = k;
      }
      unsigned msk = cand;
      while (msk && !hit) {
        const int t = __ffs(static_cast<int>(msk)) - 1;
        msk &= msk - 1u;
        const ObsRec g = obs_rec(s_pair, o0 + t);
        const float2 gx = make_float2(g.gx, g.gx), gy = make_float2(g.gy, g.gy), gz = make_float2(g.gz, g.gz),
                     gw = make_float2(g.gw, g.gw), g2 = make_float2(g.g2, g.g2);
        bool h = false;
#pragma unroll
        for (int b = 0; b < SPH_BLOCK / 2; ++b) {
          float2 v = __ffma2_rn(rs[b], g2, gw);
          v = __ffma2_rn(cz[b], gz, v);
          v = __ffma2_rn(cy[b], gy, v);
          v = __ffma2_rn(cx[b], gx, v);
          h |= (v.x < -ks[b].x) | (v.y < -ks[b].y);
        }
        tests += static_cast<uint32_t>(count);
        hit = h;
      }
    }
  }
  *tests_io = tests;
  return hit;
}

// Collision verdict of one configuration q in the collision frame: model m
// (root offsets shifted by the obstacle origin), spheres st, obstacle records
// and boxes staged in shared memory.  `tests` counts the 4-FMA tests made.
// CHUNKS: test the chunk spheres first in scenes of more than 32 obstacles
// (off where the code's size matters more than the tests it saves).
template <class P, bool CHUNKS = true>
__device__ __forceinline__ bool check_one_f32(const ModelT<float> &m, const SphereTable<float> &st,
                                              const float4 *s_pair, int n_obs, const float *s_box, int n_box,
                                              const double2 *tab, const float (&q)[P::D], uint32_t &tests) {
  const OpsF32 ops{tab};
  bool hit = false;
  {
    const Rot9 Ri{{1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f}};
    hit = link_hits_f32<CHUNKS>(Ri, V3<float>{-m.shift[0], -m.shift[1], -m.shift[2]}, st.off[0], st.off[1],
                                st.lb[MAXJ], st, s_pair, n_obs, s_box, n_box, &tests);
  }
  Kin<P, float> k;
  if (!hit)
    fk_links<P>(
        ops, m, q, k,
        [&](auto JJ, const float (&R)[9], V3<float> p) {
          constexpr int j = decltype(JJ)::value;
          if (!hit && st.off[j + 1] < st.off[j + 2]) {
            Rot9 Rr;
#pragma unroll
            for (int i = 0; i < 9; ++i) Rr.r[i] = R[i];
            hit = link_hits_f32<CHUNKS>(Rr, p, st.off[j + 1], st.off[j + 2], st.lb[j], st, s_pair, n_obs, s_box, n_box,
                                        &tests);
          }
        },
        [&]() { return hit; });
  return hit;
}

// Stages the FP32 obstacle records (in pairs, see obs_rec), the chunk
// records (in pairs, after them) and the boxes of the collision frame in
// shared memory: s_pair holds obs_pairs(n_obs) x 3 float4, then
// obs_pairs(obs_chunks(n_obs)) x 3 float4 of chunks, then the boxes.
// obs: [(n_obs + obs_chunks(n_obs)) * 8] (gx, gy, gz, gw, g2, 0, 0, 0).
__device__ __forceinline__ float *stage_obstacles(const float *obs, int n_obs, const float *box, int n_box,
                                                  float4 *s_pair) {
  const int np = obs_pairs(n_obs), nch = obs_chunks(n_obs), ncp = obs_pairs(nch);
  float *f = reinterpret_cast<float *>(s_pair);
  for (int t = threadIdx.x; t < 12 * (np + ncp); t += blockDim.x) {
    const bool chunk = t >= 12 * np;
    const int u = chunk ? t - 12 * np : t;
    const int pp = u / 12, c = u % 12, o = 2 * pp + (c & 1), field = c >> 1;  // gx gy gz gw g2 pad
    const int n = chunk ? nch : n_obs;
    const float *src = chunk ? obs + 8 * n_obs : obs;
    float v = 0.f;
    if (field < 5) v = o < n ? src[8 * o + field] : (field == 3 ? 1e30f : 0.f);  // padding: gw huge
    f[t] = v;
  }
  float *s_box = f + 12 * (np + ncp);
  for (int t = threadIdx.x; t < 6 * n_box; t += blockDim.x) s_box[t] = box[t];
  return s_box;
}

// FP32 check with a per-link broad phase: the link's bounding sphere is
// tested against the chunk spheres (scenes of more than 32 obstacles), then
// against the obstacles of the chunks it overlaps (same 4-FMA test); only the
// obstacles it overlaps are tested against the link's spheres.  The bound
// contains every sphere of the link, and a chunk's sphere every obstacle of
// the chunk, each with a 1e-4 m margin, so no overlapping pair is skipped and
// the verdict is that of the all-pairs test.  `pairs` counts every 4-FMA test
// performed (chunks, broad and narrow).
// Resident blocks of 128 threads the check asks for: trees of more than 14
// joints are capped at 128 registers (4 blocks, 16 warps per SM; the
// humanoid's check: 2.37 -> 2.15 ms per 1,048,576 configurations, its
// 142-register build allowing 12 warps); the arms' check was slower capped.
template <class P>
__host__ __device__ constexpr int check_min_blocks() {
  return P::D > 14 ? 4 : 1;
}
template <class P>
__global__ void __launch_bounds__(128, (check_min_blocks<P>())) k_check_f32(const __grid_constant__ CheckArgs<P, float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4 *s_pair = reinterpret_cast<float4 *>(smem_raw);  // 3 float4 per pair of obstacles
  const float *s_box = stage_obstacles(a.obs, a.n_obs, a.box, a.n_box, s_pair);
  __syncthreads();
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  constexpr int D = P::D;
  float q[D];
#pragma unroll
  for (int j = 0; j < D; ++j) q[j] = a.q[j * a.ld + i];
  uint32_t tests = 0;
  // a by-value copy lets the compiler read the model's compile-time-indexed
  // entries straight from the parameter bank (a reference costs registers)
  const ModelT<float> m = a.m;
  const bool hit = check_one_f32<P>(m, a.st, s_pair, a.n_obs, s_box, a.n_box, a.tab, q, tests);
  a.out[i] = hit ? 1 : 0;
  if (a.pairs) a.pairs[i] = tests;
}

template <class P>
__global__ void __launch_bounds__(128) k_check_f64(const __grid_constant__ CheckArgs<P, double> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *s_obs = reinterpret_cast<double *>(smem_raw);
  double *s_box = s_obs + 4 * a.n_obs;
  for (int t = threadIdx.x; t < 4 * a.n_obs; t += blockDim.x) s_obs[t] = a.obs[t];
  for (int t = threadIdx.x; t < 6 * a.n_box; t += blockDim.x) s_box[t] = a.box[t];
  __syncthreads();
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  constexpr int D = P::D;
  const OpsF64Plain ops{a.tab};
  double q[D];
#pragma unroll
  for (int j = 0; j < D; ++j) q[j] = a.q[j * a.ld + i];
  bool hit = false;
  uint32_t pairs = 0;
  for (int s = a.st.off[0]; s < a.st.off[1] && !hit; ++s) {
    hit = sphere_hits_plain<double>(V3<double>{a.st.s[s][0], a.st.s[s][1], a.st.s[s][2]}, a.st.s[s][3], s_obs,
                                    a.n_obs, s_box, a.n_box);
    pairs += a.n_obs;
  }
  Kin<P, double> k;
  if (!hit)
    fk_links<P>(
        ops, a.m, q, k,
        [&](auto JJ, const double (&R)[9], V3<double> p) {
          constexpr int j = decltype(JJ)::value;
          for (int s = a.st.off[j + 1]; s < a.st.off[j + 2] && !hit; ++s) {
            const V3<double> c = add_rot_t<7>(p, R, V3<double>{a.st.s[s][0], a.st.s[s][1], a.st.s[s][2]});
            hit = sphere_hits_plain<double>(c, a.st.s[s][3], s_obs, a.n_obs, s_box, a.n_box);
            pairs += a.n_obs;
          }
        },
        [&]() { return hit; });
  a.out[i] = hit ? 1 : 0;
  if (a.pairs) a.pairs[i] = pairs;
}

// ---------------------------------------------------------------------------
// Persistent projection kernel (FP32 steps, FP64 acceptance).
//
// Each warp keeps a local queue of work items claimed `chunk` at a time with
// one atomicAdd.  Every pass of the loop (1) refills idle lanes from the queue,
// (2) runs one Newton iteration on every active lane, (3) parks lanes that left
// the FP32 loop in a per-warp pending list, and (4) once 32 are pending (or no
// work is left) runs the FP64 acceptance on them with all lanes busy.  Lanes
// therefore never wait for the slowest configuration of their warp, and the
// FP64 work runs in full warps, interleaved with other warps' FP32 work.
// ---------------------------------------------------------------------------
// Register budget of the persistent kernel: what the FP32 loop needs (the FP64
// finishing path may spill; it is rare).  Sets the resident blocks per SM.
template <class P>
__host__ __device__ constexpr int reg_cap() {
  return (P::D <= 7 && kdim<P>() <= 2) ? 128 : 168;
}
template <class P, int TPB>
__host__ __device__ constexpr int min_blocks() {
  return 65536 / (TPB * reg_cap<P>()) > 0 ? 65536 / (TPB * reg_cap<P>()) : 1;
}

// Configurations a warp can hold for an FP32 retry after a failed FP64
// acceptance (beyond this the acceptance finishes them in FP64 itself).
constexpr int RETRY_CAP = 32;

template <class P, class Src, int TPB, int FORM, bool CHK>
__global__ void __launch_bounds__(TPB, (min_blocks<P, TPB>())) k_project_f32(const __grid_constant__ ProjArgs<P, Src> a) {
  constexpr int D = P::D;
  constexpr int W = TPB / 32;
  __shared__ long long s_item[W][64];
  __shared__ uint32_t s_meta[W][64];
  __shared__ long long s_ritem[W][RETRY_CAP];  // sent back to the FP32 loop by the acceptance
  __shared__ uint32_t s_rmeta[W][RETRY_CAP];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4 *s_pair = reinterpret_cast<float4 *>(smem_raw);
  const float *s_box = nullptr;
  if constexpr (CHK) {  // obstacles of the fused check, staged once per block
    s_box = stage_obstacles(a.obs, a.n_obs, a.box, a.n_box, s_pair);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const long long total = a.src.clamp_total(a.total);
  int pend = 0;                   // warp-uniform count of pending configurations
  int nret = 0;                   // warp-uniform count of configurations to retry in FP32
  long long qn = 0, qe = 0;       // warp-local queue [qn, qe)
  bool more = true;               // the global counter may still have work
  bool act = false;
  long long item = 0;
  int it = 0;
  uint32_t fl = 0;
  float q[D];
#pragma unroll
  for (int j = 0; j < D; ++j) q[j] = 0.f;

  while (true) {
    // (1) refill: configurations sent back by the acceptance first, then new work
    const unsigned idle = __ballot_sync(FULL, !act);
    if (idle != 0u && (nret > 0 || qn < qe || more)) {
      const int n_idle = __popc(idle);
      const int from_r = n_idle < nret ? n_idle : nret;
      const int need = n_idle - from_r;
      const long long avail = qe - qn;
      long long b0 = 0, b1 = 0;
      if (need > 0 && avail < need && more) {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(a.counter, static_cast<unsigned long long>(a.chunk));
        b = __shfl_sync(FULL, b, 0);
        if (static_cast<long long>(b) >= total) {
          more = false;
        } else {
          b0 = static_cast<long long>(b);
          b1 = b0 + a.chunk < total ? b0 + a.chunk : total;
        }
      }
      const int rank_all = __popc(idle & ((1u << lane) - 1u));
      if (!act) {
        if (rank_all < from_r) {  // one more FP32 step from the parked iterate
          const int pos = nret - 1 - rank_all;
          item = s_ritem[wib][pos];
          const uint32_t meta = s_rmeta[wib][pos];
          it = static_cast<int>(meta & 0xffu);
          fl = ((meta >> 8) & ~(FL_INT_FP32CONV | FL_INT_NEEDS_F64)) | FL_INT_FORCE;
          act = true;
#pragma unroll
          for (int j = 0; j < D; ++j) q[j] = MCP_CHK(item, a.ld_out) ? a.q_out[j * a.ld_out + item] : 0.f;
        } else {
          const int rank = rank_all - from_r;
          long long cand = -1;
          if (rank < avail) cand = qn + rank;
          else if (rank - avail < b1 - b0) cand = b0 + (rank - avail);
          if (cand >= 0) {
            item = cand;
            act = true;
            it = 0;
            fl = 0;
            a.src.template load<D>(item, q);
          }
        }
      }
      nret -= from_r;
      const long long used_old = need < avail ? need : avail;
      if (b1 > b0) {
        const long long rest = need - used_old;
        qn = b0 + (rest < b1 - b0 ? rest : b1 - b0);
        qe = b1;
      } else {
        qn += used_old;
      }
    }
    // (2) one FP32 Newton iteration
    bool done = false;
    if (act) {
      if constexpr (FORM == FORM_CYCLIC) done = cyclic_iter_f32<P>(a, q, it, fl);
      else done = newton_iter_f32<P, ProjArgs<P, Src>, FORM == FORM_OUTER>(a, q, it, fl);
    }
    // (3) park finished lanes
    const unsigned fin = __ballot_sync(FULL, done);
    if (fin != 0u) {
      if (done) {
        if (MCP_CHK(item, a.ld_out)) {
#pragma unroll
          for (int j = 0; j < D; ++j) a.q_out[j * a.ld_out + item] = q[j];
        }
        const int pos = pend + __popc(fin & ((1u << lane) - 1u));
        s_item[wib][pos] = item;
        s_meta[wib][pos] = static_cast<uint32_t>(it) | (fl << 8);
        act = false;
      }
      pend += __popc(fin);
      __syncwarp();
    }
    const bool drained = !__any_sync(FULL, act) && qn >= qe && !more && nret == 0;
    // (4) FP64 acceptance in full warps (and, fused, the collision check of
    // the accepted outputs: ALU work that overlaps other warps' FP64 passes);
    // a failed acceptance with steps left is queued for one more FP32 step
    // (an FP64 step on one lane would hold the FP64 pipe as long as 32 lanes)
    if (pend >= 32 || (drained && pend > 0)) {
      const int take = pend < 32 ? pend : 32;
      const bool room = nret + take <= RETRY_CAP;
      bool retry = false;
      long long it_item = 0;
      uint32_t meta = 0;
      if (lane < take) {
        const int pos = pend - take + lane;
        meta = s_meta[wib][pos];
        it_item = s_item[wib][pos];
        retry = accept_one<P, FORM>(a, it_item, static_cast<int>(meta & 0xffu), meta >> 8, room);
        if constexpr (CHK) {
          if (!retry) {
            float qc[D];
            const bool okc = MCP_CHK(it_item, a.ld_out);
#pragma unroll
            for (int j = 0; j < D; ++j) qc[j] = okc ? a.q_out[j * a.ld_out + it_item] : 0.f;
            uint32_t tests = 0;
            const bool h = check_one_f32<P>(a.chk->m, a.chk->st, s_pair, a.n_obs, s_box, a.n_box, a.tab, qc, tests);
            if (okc) a.hit[it_item] = h ? 1 : 0;
            if (a.pairs) a.pairs[it_item] = tests;
          }
        }
      }
      const unsigned rm = __ballot_sync(FULL, retry);
      __syncwarp();
      if (retry) {
        const int rp = nret + __popc(rm & ((1u << lane) - 1u));
        s_ritem[wib][rp] = it_item;
        s_rmeta[wib][rp] = meta;
      }
      nret += __popc(rm);
      pend -= take;
      __syncwarp();
    }
    if (drained && pend == 0 && nret == 0) break;
  }
}

// ---------------------------------------------------------------------------
// Plain FP64 kernel: one thread per configuration, FP64 and CUDA's double
// math throughout, no staging, no refill.  The reference point the batched
// FP32 path is measured against, and the product path of FP64 problems.
// ---------------------------------------------------------------------------
template <class P, class Src>
struct ProjArgs64 {
  ModelT<double> m;
  Src src;
  double *q_out;
  long long ld_out;
  uint8_t *flags;
  uint8_t *iters;
  double *resid;
  long long total;
  int cap;
  double tol2;
  double lambda;
  double max_step2;
  double alpha;
};

// One plain FP64 LM step of the (sub-)problem S at q: dq = J^T (J J^T + lambda I)^-1 F.
// Returns false if the system is singular.
template <class S, class M, bool OUTER = false>
__device__ __forceinline__ bool step_f64(const M &m, const double (&q)[S::D], double lambda, double (&dq)[S::D]) {
  constexpr int D = S::D, K = kdim<S>();
  const OpsF64Plain ops{nullptr};
  Kin<S, double> k;
  if constexpr (needs_fk<S>()) fk<S, needs_pos<S>()>(ops, m, q, k);
  double F[K];
  Eval<S, double> e;
  residual<S, OpsF64Plain, double, true>(m, q, k, F, e);
  double J[K][D];
  jacobian<S>(m, q, k, e, J);
  if constexpr (OUTER) {
    double Am[D * (D + 1) / 2];
    gram_outer<S>(J, lambda, Am);
    jt_mul<S>(J, F, dq);
    return cholesky_solve<D, OpsF64Plain>(Am, dq) > 0.0;
  } else {
    double Am[K * (K + 1) / 2];
    gram<S>(J, lambda, Am);
    const double piv = cholesky_solve<K, OpsF64Plain>(Am, F);
    if (!(piv > 0.0)) return false;
    jt_mul<S>(J, F, dq);
    return true;
  }
}

template <class P, class Src, int FORM>
__global__ void __launch_bounds__(128) k_project_f64(const __grid_constant__ ProjArgs64<P, Src> a) {
  constexpr int D = P::D, K = kdim<P>();
  constexpr bool CYC = FORM == FORM_CYCLIC;
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.src.clamp_total(a.total)) return;
  const OpsF64Plain ops{nullptr};
  double q[D];
  a.src.template load<D>(i, q);
  uint32_t fl = 0;
  int it = 0;
  double r2 = 0.0;
  for (;; ++it) {
    Kin<P, double> k;
    if constexpr (needs_fk<P>()) fk<P, needs_pos<P>()>(ops, a.m, q, k);
    double F[K];
    Eval<P, double> e;
    residual<P, OpsF64Plain, double, !CYC>(a.m, q, k, F, e);
    r2 = 0.0;
#pragma unroll
    for (int r = 0; r < K; ++r) r2 = fma(F[r], F[r], r2);
    if (!(r2 <= DBL_MAX)) {
      fl |= FL_NONFINITE;
      break;
    }
    if (r2 < a.tol2) {
      fl |= FL_CONV;
      break;
    }
    if (it >= a.cap) {
      fl |= FL_CAP;
      break;
    }
    if constexpr (CYC) {
      // cyclic getDescentStep (Sec. IV-C): one step per constraint, in order
      double q0[D];
#pragma unroll
      for (int j = 0; j < D; ++j) q0[j] = q[j];
      bool sing = false;
      static_for<P::NC>([&](auto CC) {
        if (sing) return;
        double dq[D];
        if (!step_f64<Sub<P, decltype(CC)::value>>(a.m, q, a.lambda, dq)) {
          sing = true;
          return;
        }
#pragma unroll
        for (int j = 0; j < D; ++j) q[j] -= a.alpha * dq[j];
      });
      if (sing) {
        fl |= FL_NONFINITE;
        break;
      }
      double s2 = 0.0;
#pragma unroll
      for (int j = 0; j < D; ++j) s2 = fma(q[j] - q0[j], q[j] - q0[j], s2);
      if (a.max_step2 > 0.0 && s2 > a.max_step2) {
#pragma unroll
        for (int j = 0; j < D; ++j) q[j] = q0[j];
        fl |= FL_DIV;
        break;
      }
    } else {
      double J[K][D];
      jacobian<P>(a.m, q, k, e, J);
      double dq[D];
      double piv;
      if constexpr (FORM == FORM_OUTER) {
        double Am[D * (D + 1) / 2];
        gram_outer<P>(J, a.lambda, Am);
        jt_mul<P>(J, F, dq);
        piv = cholesky_solve<D, OpsF64Plain>(Am, dq);
      } else {
        double Am[K * (K + 1) / 2];
        gram<P>(J, a.lambda, Am);
        piv = cholesky_solve<K, OpsF64Plain>(Am, F);
        jt_mul<P>(J, F, dq);
      }
      if (!(piv > 0.0)) {
        fl |= FL_NONFINITE;
        break;
      }
      double s2 = 0.0;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        dq[j] *= a.alpha;
        s2 = fma(dq[j], dq[j], s2);
      }
      if (a.max_step2 > 0.0 && s2 > a.max_step2) {
        fl |= FL_DIV;
        break;
      }
#pragma unroll
      for (int j = 0; j < D; ++j) q[j] -= dq[j];
    }
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    a.q_out[j * a.ld_out + i] = q[j];
    if (q[j] < a.m.lower[j] || q[j] > a.m.upper[j]) fl |= FL_LIMITS;
  }
  a.flags[i] = static_cast<uint8_t>(fl);
  a.iters[i] = static_cast<uint8_t>(it > 255 ? 255 : it);
  a.resid[i] = sqrt(r2);
}

// ---------------------------------------------------------------------------
// VJP of the projection at q* (implicit-function theorem):
//     v = g - J^T (J J^T)^{-1} J g.
// FP32 with the same pivot rule as the projection: a small pivot re-solves
// the configuration in FP64.
// ---------------------------------------------------------------------------
template <class P>
struct VjpArgs {
  ModelT<float> m;
  const ModelT<double> *__restrict__ m64;
  const double2 *__restrict__ tab;
  const float *q;
  const float *g;
  float *out;
  uint8_t *flags;
  long long ld;
  long long n;
  float pivot;
};

template <class P>
__device__ __noinline__ uint32_t vjp_f64(const OpsF64Table ops, const ModelT<double> *__restrict__ m,
                                          const double *q, const double *g, double *v) {
  // Reuse the FP64 LM step: with F replaced by J g and lambda = 0 it returns
  // J^T (J J^T)^{-1} J g.  lm_step_f64 evaluates F itself, so the product is
  // formed here instead.
  constexpr int D = P::D, K = kdim<P>();
  double qq[D];
#pragma unroll
  for (int j = 0; j < D; ++j) qq[j] = q[j];
  Kin<P, double> k;
  if constexpr (needs_fk<P>()) fk<P, needs_pos<P>()>(ops, *m, qq, k);
  double F[K];
  Eval<P, double> e;
  residual<P, OpsF64Table, double, true>(*m, qq, k, F, e);
  double J[K][D];
#pragma unroll 1
  for (int a = 0; a < K; ++a)
#pragma unroll 1
    for (int j = 0; j < D; ++j) J[a][j] = 0.0;
  jacobian<P>(*m, qq, k, e, J);
  double L[K][K], u[K];
#pragma unroll 1
  for (int a = 0; a < K; ++a) {
    double s = 0.0;
#pragma unroll 1
    for (int j = 0; j < D; ++j) s = fma(J[a][j], g[j], s);
    u[a] = s;
#pragma unroll 1
    for (int b = 0; b <= a; ++b) {
      double t = 0.0;
#pragma unroll 1
      for (int j = 0; j < D; ++j) t = fma(J[a][j], J[b][j], t);
      L[a][b] = t;
    }
  }
#pragma unroll 1
  for (int j = 0; j < K; ++j) {
    double s = L[j][j];
#pragma unroll 1
    for (int t = 0; t < j; ++t) s = fma(-L[j][t], L[j][t], s);
    if (!(s > 0.0)) return FL_NONFINITE;
    L[j][j] = sqrt(s);
#pragma unroll 1
    for (int i = j + 1; i < K; ++i) {
      double t2 = L[i][j];
#pragma unroll 1
      for (int t = 0; t < j; ++t) t2 = fma(-L[i][t], L[j][t], t2);
      L[i][j] = t2 / L[j][j];
    }
  }
#pragma unroll 1
  for (int i = 0; i < K; ++i) {
    double s = u[i];
#pragma unroll 1
    for (int t = 0; t < i; ++t) s = fma(-L[i][t], u[t], s);
    u[i] = s / L[i][i];
  }
#pragma unroll 1
  for (int i = K - 1; i >= 0; --i) {
    double s = u[i];
#pragma unroll 1
    for (int t = i + 1; t < K; ++t) s = fma(-L[t][i], u[t], s);
    u[i] = s / L[i][i];
  }
#pragma unroll 1
  for (int j = 0; j < D; ++j) {
    double s = 0.0;
#pragma unroll 1
    for (int a = 0; a < K; ++a) s = fma(J[a][j], u[a], s);
    v[j] = g[j] - s;
  }
  return FL_RESOLVE;
}

template <class P>
// 128 registers (4 blocks per SM): 65,536 VJPs in one wave of blocks; at
// 252 registers (no spills) they took two waves and 8 % longer.
__global__ void __launch_bounds__(128, 4) k_vjp(const __grid_constant__ VjpArgs<P> a) {
  constexpr int D = P::D, K = kdim<P>();
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const OpsF32 ops{a.tab};
  float q[D], g[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    q[j] = a.q[j * a.ld + i];
    g[j] = a.g[j * a.ld + i];
  }
  Kin<P, float> k;
  if constexpr (needs_fk<P>()) fk<P, needs_pos<P>()>(ops, a.m, q, k);
  float F[K];
  Eval<P, float> e;
  residual<P, OpsF32, float, true>(a.m, q, k, F, e);
  float J[K][D];
  jacobian<P>(a.m, q, k, e, J);
  float Am[K * (K + 1) / 2], inv[K];
  gram<P>(J, 0.f, Am);
  float u[K], y[K], w0[D];
  j_mul<P>(J, g, u);
  const float piv = cholesky_factor<K, OpsF32>(Am, inv);
#pragma unroll
  for (int i = 0; i < K; ++i) y[i] = u[i];
  cholesky_subst<K>(Am, inv, y);
  jt_mul<P>(J, y, w0);
  refine_step<P>(J, u, 0.f, Am, inv, y, w0);
  uint32_t fl = 0;
  if (!(piv >= a.pivot)) {
    double qd[D], gd[D], vd[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      qd[j] = q[j];
      gd[j] = g[j];
    }
    fl = vjp_f64<P>(OpsF64Table{a.tab}, a.m64, qd, gd, vd);
#pragma unroll
    for (int j = 0; j < D; ++j) a.out[j * a.ld + i] = (fl & FL_NONFINITE) ? CUDART_NAN_F : static_cast<float>(vd[j]);
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j) a.out[j * a.ld + i] = g[j] - w0[j];
  }
  if (a.flags) a.flags[i] = static_cast<uint8_t>(fl);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <class P, class Src, int TPB, int FORM, bool CHK>
cudaError_t launch_persistent(const HostModel &hm, const ProjCall &c, const Src &src) {
  ProjArgs<P, Src> a;
  a.m = hm.m32;
  a.m64 = hm.d_m64;
  a.tab = hm.d_tab;
  a.src = src;
  a.q_out = static_cast<float *>(c.q_out);
  a.ld_out = c.ld_out;
  a.flags = c.flags;
  a.iters = c.iters;
  a.resid = c.resid;
  a.counter = c.counter;
  a.total = c.total;
  a.chunk = c.tune.chunk;
  a.cap = c.cap;
  a.tol2 = static_cast<float>(c.tol * c.tol);
  a.lambda = static_cast<float>(c.lambda);
  a.max_step2 = c.max_step > 0 ? static_cast<float>(c.max_step * c.max_step) : 0.f;
  a.pivot = static_cast<float>(c.pivot);
  a.tol2_64 = c.tol * c.tol;
  a.lambda64 = c.lambda;
  a.alpha = static_cast<float>(c.alpha);
  a.chk = hm.d_chk;
  a.obs = reinterpret_cast<const float *>(hm.d_obs32);
  a.box = hm.d_box32;
  a.n_obs = CHK ? hm.n_obs : 0;
  a.n_box = CHK ? hm.n_box : 0;
  a.hit = c.hit;
  a.pairs = c.pairs;
  const size_t smem = CHK ? obs_smem_bytes(hm.n_obs, hm.n_box) : 0;
  const long long warps_needed = (c.total + 31) / 32;
  long long blocks = static_cast<long long>(hm.sm_count) * c.tune.blocks_per_sm;
  const long long max_useful = (warps_needed + (TPB / 32) - 1) / (TPB / 32);
  if (blocks > max_useful) blocks = max_useful;
  if (blocks < 1) blocks = 1;
  k_project_f32<P, Src, TPB, FORM, CHK><<<static_cast<unsigned>(blocks), TPB, smem, c.stream>>>(a);
  return cudaGetLastError();
}

template <class P, class Src, int FORM = FORM_STACKED>
cudaError_t launch_plain64(const HostModel &hm, const ProjCall &c, const Src &src) {
  ProjArgs64<P, Src> a;
  a.m = hm.m64;
  a.src = src;
  a.q_out = static_cast<double *>(c.q_out);
  a.ld_out = c.ld_out;
  a.flags = c.flags;
  a.iters = c.iters;
  a.resid = c.resid;
  a.total = c.total;
  a.cap = c.cap;
  a.tol2 = c.tol * c.tol;
  a.lambda = c.lambda;
  a.max_step2 = c.max_step > 0 ? c.max_step * c.max_step : 0.0;
  a.alpha = c.alpha;
  const long long blocks = (c.total + 127) / 128;
  k_project_f64<P, Src, FORM><<<static_cast<unsigned>(blocks), 128, 0, c.stream>>>(a);
  return cudaGetLastError();
}

// Plain FP64 launch in the requested form (one constraint: cyclic = stacked).
template <class P, class Src>
cudaError_t launch_plain64_any(const HostModel &hm, const ProjCall &c, const Src &src) {
  if (c.outer) {
    if constexpr (P::D <= 14) return launch_plain64<P, Src, FORM_OUTER>(hm, c, src);
    else return cudaErrorNotSupported;
  }
  if constexpr (P::NC > 1) {
    if (c.cyclic) return launch_plain64<P, Src, FORM_CYCLIC>(hm, c, src);
  }
  return launch_plain64<P, Src, FORM_STACKED>(hm, c, src);
}

template <class P>
cudaError_t launch_check_impl(const HostModel &hm, const CheckCall &c, int *launches);

// The collision check of a projection's outputs as a launch of its own (paths
// without a fused kernel): same verdicts as check_batch on q_out.
template <class P>
cudaError_t check_outputs(const HostModel &hm, const ProjCall &c, int *launches) {
  CheckCall cc;
  cc.precision = c.precision;
  cc.n = c.total;
  cc.ld = c.ld_out;
  cc.q = c.q_out;
  cc.out = c.hit;
  cc.pairs = c.pairs;
  cc.stream = c.stream;
  return launch_check_impl<P>(hm, cc, launches);
}

template <class P>
cudaError_t launch_project_impl(const HostModel &hm, const ProjCall &c, int *launches) {
  if (c.total <= 0) return cudaSuccess;
  cudaError_t err;
  if (c.precision == 1) {
    if (c.segments)
      err = launch_plain64_any<P>(hm, c, SegSrc<double>{static_cast<const double *>(c.start),
                                                        static_cast<const double *>(c.delta), c.ld_seg,
                                                        c.seg_off, c.n_seg});
    else
      err = launch_plain64_any<P>(hm, c, BatchSrc<double>{static_cast<const double *>(c.q_in), c.ld_in});
    *launches += 1;
    if (err == cudaSuccess && c.fused_check) err = check_outputs<P>(hm, c, launches);
    return err;
  }
  err = cudaMemsetAsync(c.counter, 0, sizeof(unsigned long long), c.stream);
  if (err != cudaSuccess) return err;
  auto go = [&](auto src, auto chk) -> cudaError_t {
    using S = decltype(src);
    constexpr bool CHK = decltype(chk)::value;
    if (c.outer) {  // the outer form: d x d systems, thread kernels up to 14 joints
      if constexpr (P::D <= 14 && !CHK && std::is_same_v<S, BatchSrc<float>>)
        return launch_persistent<P, S, 128, FORM_OUTER, false>(hm, c, src);
      else
        return cudaErrorNotSupported;
    }
    if constexpr (P::NC > 1) {  // one constraint: the cyclic and stacked forms coincide
      if (c.cyclic) return launch_persistent<P, S, 128, FORM_CYCLIC, CHK>(hm, c, src);
    }
    switch (c.tune.tpb) {
      case 64: return launch_persistent<P, S, 64, FORM_STACKED, CHK>(hm, c, src);
      case 256: return launch_persistent<P, S, 256, FORM_STACKED, CHK>(hm, c, src);
      default: return launch_persistent<P, S, 128, FORM_STACKED, CHK>(hm, c, src);
    }
  };
  if (c.segments) {
    err = go(SegSrc<float>{static_cast<const float *>(c.start), static_cast<const float *>(c.delta), c.ld_seg,
                           c.seg_off, c.n_seg},
             std::false_type{});
    *launches += 1;
    if (err == cudaSuccess && c.fused_check) err = check_outputs<P>(hm, c, launches);
    return err;
  }
  const BatchSrc<float> src{static_cast<const float *>(c.q_in), c.ld_in};
  err = c.fused_check ? go(src, std::true_type{}) : go(src, std::false_type{});
  *launches += 1;
  return err;
}

template <class P>
cudaError_t launch_check_impl(const HostModel &hm, const CheckCall &c, int *launches) {
  if (c.n <= 0) return cudaSuccess;
  const unsigned blocks = static_cast<unsigned>((c.n + 127) / 128);
  if (c.precision == 1) {
    CheckArgs<P, double> a;
    a.m = hm.m64;
    a.st = hm.st64;
    a.obs = hm.d_obs64;
    a.box = hm.d_box64;
    a.n_obs = hm.n_obs;
    a.n_box = hm.n_box;
    a.q = static_cast<const double *>(c.q);
    a.ld = c.ld;
    a.n = c.n;
    a.out = c.out;
    a.pairs = c.pairs;
    a.tab = hm.d_tab;
    const size_t smem = sizeof(double) * (4 * hm.n_obs + 6 * hm.n_box);
    k_check_f64<P><<<blocks, 128, smem, c.stream>>>(a);
  } else {
    CheckArgs<P, float> a;
    a.m = hm.m32_shifted;
    a.st = hm.st32;
    a.obs = reinterpret_cast<const float *>(hm.d_obs32);
    a.box = reinterpret_cast<const float *>(hm.d_box32);
    a.n_obs = hm.n_obs;
    a.n_box = hm.n_box;
    a.q = static_cast<const float *>(c.q);
    a.ld = c.ld;
    a.n = c.n;
    a.out = c.out;
    a.pairs = c.pairs;
    a.tab = hm.d_tab;
    const size_t smem = obs_smem_bytes(hm.n_obs, hm.n_box);
    k_check_f32<P><<<blocks, 128, smem, c.stream>>>(a);
  }
  *launches += 1;
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_vjp_impl(const HostModel &hm, const VjpCall &c, int *launches) {
  if (c.n <= 0) return cudaSuccess;
  VjpArgs<P> a;
  a.m = hm.m32;
  a.m64 = hm.d_m64;
  a.tab = hm.d_tab;
  a.q = c.q;
  a.g = c.g;
  a.out = c.out;
  a.flags = c.flags;
  a.ld = c.ld;
  a.n = c.n;
  a.pivot = static_cast<float>(c.pivot);
  const unsigned blocks = static_cast<unsigned>((c.n + 127) / 128);
  k_vjp<P><<<blocks, 128, 0, c.stream>>>(a);
  *launches += 1;
  return cudaGetLastError();
}

#define MCP_NO_EXTEND(P)                                                                       \
  template <>                                                                                  \
  cudaError_t launch_extend<P>(const HostModel &, const ExtCall &, int *) {                     \
    return cudaErrorNotSupported;                                                              \
  }

#define MCP_INSTANTIATE_CHECK_ONLY(P)                                                          \
  template <>                                                                                  \
  cudaError_t launch_project<P>(const HostModel &, const ProjCall &, int *) {                   \
    return cudaErrorNotSupported;                                                              \
  }                                                                                            \
  template <>                                                                                  \
  cudaError_t launch_check<P>(const HostModel &hm, const CheckCall &c, int *launches) {        \
    return launch_check_impl<P>(hm, c, launches);                                              \
  }                                                                                            \
  template <>                                                                                  \
  cudaError_t launch_vjp<P>(const HostModel &, const VjpCall &, int *) {                        \
    return cudaErrorNotSupported;                                                              \
  }

#define MCP_INSTANTIATE(P)                                                                     \
  template <>                                                                                  \
  cudaError_t launch_project<P>(const HostModel &hm, const ProjCall &c, int *launches) {       \
    return launch_project_impl<P>(hm, c, launches);                                            \
  }                                                                                            \
  template <>                                                                                  \
  cudaError_t launch_check<P>(const HostModel &hm, const CheckCall &c, int *launches) {        \
    return launch_check_impl<P>(hm, c, launches);                                              \
  }                                                                                            \
  template <>                                                                                  \
  cudaError_t launch_vjp<P>(const HostModel &hm, const VjpCall &c, int *launches) {            \
    return launch_vjp_impl<P>(hm, c, launches);                                                \
  }

}  // namespace mcp
