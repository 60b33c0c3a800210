// Warp-cooperative projection for large problem classes (the 36-DoF humanoid
// with 20 stacked equations), where one configuration's Jacobian (K x D) and
// Gram matrix do not fit one thread's registers.
//
// One warp owns one configuration at a time; its state lives in shared memory.
// Per FP32 iteration of Alg. 2 (stacked F, inner LM form):
//   1. local transforms L_j = X_j Jnt(q_j), one joint per lane;
//   2. world transforms by a parallel prefix over the tree (pointer jumping:
//      T_j <- T_anc(j) T_j, anc(j) <- anc(anc(j)), ceil(log2(depth)) rounds);
//   3. task frames, link CoMs, subtree CoM sums (joints are in depth-first
//      order, so a subtree is a contiguous index range);
//   4. residuals, one constraint per lane; ||F|| by a warp reduction;
//   5. Jacobian columns, one joint per lane;
//   6. Gram rows, one row per lane, J rows read with broadcast loads;
//   7. right-looking Cholesky with one matrix row per lane (registers),
//      forward / back substitution, dq = J^T y, one joint per lane.
// Finished configurations are parked; once 32 are parked, the FP64
// acceptance runs one configuration per lane (the thread-level FP64 code).
#pragma once

#include "mcp_kernels.cuh"

namespace mcp {

template <class P>
struct WarpTables {
  float X[P::D][12];
  float mass[P::D];
  float com[P::D][4];
  float msub[P::D];
  int parent[P::D];
  int rev[P::D];
  int sub_end[P::D];         // subtree of j = joints [j, sub_end[j])
  float coef[P::NC][P::D];   // column sign of joint j in constraint c (0, +1, -1)
  float fX[P::NF][12];
};

template <class P>
__host__ __device__ constexpr int tree_depth() {
  int best = 0;
  for (int j = 0; j < P::D; ++j) {
    int d = 0;
    for (int l = j; l >= 0; l = P::parent(l)) ++d;
    best = d > best ? d : best;
  }
  return best;
}
__host__ __device__ constexpr int ceil_log2(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}
template <class P>
__host__ __device__ constexpr bool dfs_preorder() {
  // every joint's parent precedes it and each subtree is a contiguous range
  for (int j = 0; j < P::D; ++j) {
    if (P::parent(j) >= j) return false;
    int end = j + 1;
    while (end < P::D && is_anc<P>(j, end)) ++end;
    for (int i = end; i < P::D; ++i)
      if (is_anc<P>(j, i)) return false;
  }
  return true;
}

// Block structure of J for the Gram build: the float4 groups of rows that
// hold a structural nonzero in column j, and the runs of consecutive joints
// with the same groups (in depth-first order a limb is one run).
template <class P>
__host__ __device__ constexpr unsigned col_groups(int j) {
  unsigned g = 0;
  for (int r = 0; r < kdim<P>(); ++r)
    if (jnz<P>(r, j)) g |= 1u << (r / 4);
  return g;
}
template <class P>
struct GramRuns {
  int n;
  int begin[P::D + 1];
  unsigned mask[P::D];
};
template <class P>
__host__ __device__ constexpr GramRuns<P> gram_runs() {
  GramRuns<P> g{};
  g.n = 0;
  for (int j = 0; j < P::D; ++j) {
    const unsigned m = col_groups<P>(j);
    if (g.n == 0 || g.mask[g.n - 1] != m) {
      g.begin[g.n] = j;
      g.mask[g.n] = m;
      ++g.n;
    }
  }
  g.begin[g.n] = P::D;
  return g;
}
// Does constraint c have a structurally nonzero column among joints [j0, j1)?
template <class P>
__host__ __device__ constexpr bool any_column(int c, int j0, int j1) {
  for (int j = j0; j < j1 && j < P::D; ++j)
    if (col_sign<P>(c, j) != 0) return true;
  return false;
}

template <class P>
struct __align__(16) WarpState {
  static constexpr int D = P::D, K = kdim<P>(), KP = (kdim<P>() + 3) & ~3;
  float T[D][12];
  float J[D][KP];
  float L[K][KP];
  float F[KP];
  float y[KP];
  float Tf[P::NF][12];
  float mc[D][4];   // m_j c_j
  float C[D][4];    // subtree sums
  float q[D];
  float dq[D];
  float q0[D];      // start of a cyclic sweep
  int anc[D];
  float G[P::NC][9];
  float x[P::NC][4];
  float phi[P::NC][4];
  float beta[P::NC];
  float za[P::NC][4];
  float hn[P::NC][2];  // support-hull constraint: normal of the nearest edge
  int hmode[P::NC];    // 0 inside, 1 on an edge, 2 at a vertex
};

template <class P>
struct WarpArgs {
  ModelT<float> m;
  WarpTables<P> t;
  const ModelT<double> *__restrict__ m64;
  const double2 *__restrict__ tab;
  BatchSrc<float> src;
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
  float alpha;
};

// C = A B for row-major 3x4 rigid transforms held in registers
__device__ __forceinline__ void compose34(const float (&A)[12], const float (&B)[12], float (&C)[12]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      C[r * 4 + c] = fmaf(A[r * 4], B[c], fmaf(A[r * 4 + 1], B[4 + c], A[r * 4 + 2] * B[8 + c]));
    C[r * 4 + 3] = fmaf(A[r * 4], B[3], fmaf(A[r * 4 + 1], B[7], fmaf(A[r * 4 + 2], B[11], A[r * 4 + 3])));
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Modes of warp_iter: one stacked iteration; only the stopping test on the
// stacked F (the head of a cyclic sweep); or (MODE = c >= 0) the LM step of
// constraint c alone, with the rows of the other constraints masked out of F
// and J and given a unit diagonal, which decouples them exactly.
constexpr int WI_STACKED = -2, WI_CHECK = -1;

// One FP32 iteration on the warp's configuration.  Returns true when the
// configuration leaves the FP32 loop (flags say why).
template <class P, int MODE, class A>
__device__ __forceinline__ bool warp_iter(const A &a, const WarpTables<P> &tb, WarpState<P> &S, int &it,
                                          uint32_t &fl) {
  constexpr int D = P::D, K = kdim<P>(), KP = WarpState<P>::KP;
  constexpr int SL = (D + 31) / 32;
  constexpr int ROUNDS = ceil_log2(tree_depth<P>());
  static_assert(K <= 32, "one Gram row per lane");
  const int lane = threadIdx.x & 31;
  const ModelT<float> &m = a.m;

  // 1. local transforms
  float Tc[SL][12];
  int an[SL];
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int j = lane + 32 * s;
    an[s] = -1;
    if (j < D) {
      const float *X = tb.X[j];
      const float qj = S.q[j];
      if (tb.rev[j]) {
        float sn, cs;
        sincos_f32(qj, sn, cs);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          Tc[s][r * 4] = fmaf(cs, X[r * 4], sn * X[r * 4 + 1]);
          Tc[s][r * 4 + 1] = fmaf(cs, X[r * 4 + 1], -(sn * X[r * 4]));
          Tc[s][r * 4 + 2] = X[r * 4 + 2];
          Tc[s][r * 4 + 3] = X[r * 4 + 3];
        }
      } else {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
#pragma unroll
          for (int c = 0; c < 3; ++c) Tc[s][r * 4 + c] = X[r * 4 + c];
          Tc[s][r * 4 + 3] = fmaf(qj, X[r * 4 + 2], X[r * 4 + 3]);
        }
      }
      an[s] = tb.parent[j];
#pragma unroll
      for (int e = 0; e < 12; ++e) S.T[j][e] = Tc[s][e];
      S.anc[j] = an[s];
    }
  }
  __syncwarp();
  // 2. tree prefix (pointer jumping)
#pragma unroll 1
  for (int r = 0; r < ROUNDS; ++r) {
    int an2[SL];
    float Tn[SL][12];
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      an2[s] = an[s];
      if (an[s] >= 0) {
        float Ta[12];
#pragma unroll
        for (int e = 0; e < 12; ++e) Ta[e] = S.T[an[s]][e];
        compose34(Ta, Tc[s], Tn[s]);
        an2[s] = S.anc[an[s]];
      }
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int j = lane + 32 * s;
      if (an[s] >= 0) {
#pragma unroll
        for (int e = 0; e < 12; ++e) {
          Tc[s][e] = Tn[s][e];
          S.T[j][e] = Tn[s][e];
        }
        S.anc[j] = an2[s];
        an[s] = an2[s];
      }
    }
    __syncwarp();
  }
  // 3. frames and link CoMs
  if (lane < P::NF) {
    const int f = lane;
    float Tl[12], Fx[12], To[12];
    int l = -1;
    static_for<P::NF>([&](auto FF) {
      if (decltype(FF)::value == f) l = P::frame_link(decltype(FF)::value);
    });
#pragma unroll
    for (int e = 0; e < 12; ++e) {
      Tl[e] = S.T[l][e];
      Fx[e] = tb.fX[f][e];
    }
    compose34(Tl, Fx, To);
#pragma unroll
    for (int e = 0; e < 12; ++e) S.Tf[f][e] = To[e];
  }
  float mcv[SL][3];
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int j = lane + 32 * s;
    mcv[s][0] = mcv[s][1] = mcv[s][2] = 0.f;
    if (j < D) {
      const float *c = tb.com[j];
#pragma unroll
      for (int r = 0; r < 3; ++r)
        mcv[s][r] = tb.mass[j] * fmaf(Tc[s][r * 4], c[0], fmaf(Tc[s][r * 4 + 1], c[1], fmaf(Tc[s][r * 4 + 2], c[2], Tc[s][r * 4 + 3])));
    }
  }
  // total CoM moment (warp reduction) and, per joint, the sum over its subtree
  // [j, sub_end[j]) added directly (a difference of prefix sums would lose
  // digits to cancellation for small distal subtrees)
  float tot[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float v = 0.f;
#pragma unroll
    for (int s = 0; s < SL; ++s) v += mcv[s][r];
    tot[r] = warp_sum(v);
  }
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int j = lane + 32 * s;
    if (j < D) {
      S.mc[j][0] = mcv[s][0];
      S.mc[j][1] = mcv[s][1];
      S.mc[j][2] = mcv[s][2];
    }
  }
  __syncwarp();
  if constexpr (needs_com<P>()) {
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int j = lane + 32 * s;
      if (j < D) {
        float c0 = 0.f, c1 = 0.f, c2 = 0.f;
        for (int i = j; i < tb.sub_end[j]; ++i) {
          c0 += S.mc[i][0];
          c1 += S.mc[i][1];
          c2 += S.mc[i][2];
        }
        S.C[j][0] = c0;
        S.C[j][1] = c1;
        S.C[j][2] = c2;
      }
    }
  }
  // 4. residuals: constraint c on lane c
  static_for<P::NC>([&](auto CC) {
    constexpr int c = decltype(CC)::value;
    constexpr int kind = P::ckind(c);
    constexpr int r0 = roff<P>(c);
    static_assert(kind == K_AXIS || kind == K_COM || kind == K_HULL || kind == K_POSE || kind == K_REL,
                  "the warp kernel implements the axis, CoM, CoM-hull, pose and relative-pose constraints");
    if (lane == c) {
      if constexpr (MODE >= 0 && c != MODE) {
#pragma unroll
        for (int r = 0; r < cdim(kind); ++r) S.F[r0 + r] = 0.f;
      } else if constexpr (kind == K_AXIS) {
        constexpr int fa = P::cfa(c);
        S.za[c][0] = S.Tf[fa][2];
        S.za[c][1] = S.Tf[fa][6];
        S.za[c][2] = S.Tf[fa][10];
        S.F[r0] = S.Tf[fa][2];
        S.F[r0 + 1] = S.Tf[fa][6];
      } else if constexpr (kind == K_COM) {
        S.F[r0] = fmaf(tot[0], m.inv_mass, -m.ctgt[c][0]);
        S.F[r0 + 1] = fmaf(tot[1], m.inv_mass, -m.ctgt[c][1]);
      } else if constexpr (kind == K_HULL) {
        const float cx = tot[0] * m.inv_mass, cy = tot[1] * m.inv_mass;
        float px, py, nx, ny;
        S.hmode[c] = polygon_nearest<float>(m.cB[c], static_cast<int>(m.ctgt[c][0]), cx, cy, px, py, nx, ny);
        S.hn[c][0] = nx;
        S.hn[c][1] = ny;
        S.F[r0] = cx - px;
        S.F[r0 + 1] = cy - py;
      } else {
        float Pr[9], Rerr[9], G[9];
        load_R(m.cPinv[c], Pr);
        const V3<float> Pp = load_p(m.cPinv[c]);
        V3<float> t, xpt;
        constexpr int fa = P::cfa(c);
        float Ra[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) Ra[r * 3 + cc] = S.Tf[fa][r * 4 + cc];
        const V3<float> pa{S.Tf[fa][3], S.Tf[fa][7], S.Tf[fa][11]};
        if constexpr (kind == K_POSE) {
          float Qr[9], RaQ[9];
          load_R(m.cQinv[c], Qr);
          mul33(Ra, Qr, RaQ);
          xpt = add_rot_t<7>(pa, Ra, load_p(m.cQinv[c]));
          mul33(Pr, RaQ, Rerr);
          const V3<float> tx = mulv(Pr, xpt);
          t = {tx.x + Pp.x, tx.y + Pp.y, tx.z + Pp.z};
#pragma unroll
          for (int i = 0; i < 9; ++i) G[i] = Pr[i];
        } else {
          constexpr int fb = P::cfb(c);
          float Rb[9];
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) Rb[r * 3 + cc] = S.Tf[fb][r * 4 + cc];
          const V3<float> pb{S.Tf[fb][3], S.Tf[fb][7], S.Tf[fb][11]};
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
              G[r * 3 + cc] = fmaf(Pr[r * 3], Ra[cc * 3], fmaf(Pr[r * 3 + 1], Ra[cc * 3 + 1], Pr[r * 3 + 2] * Ra[cc * 3 + 2]));
          mul33(G, Rb, Rerr);
          const V3<float> tx = mulv(G, sub(pb, pa));
          t = {tx.x + Pp.x, tx.y + Pp.y, tx.z + Pp.z};
          xpt = pb;
        }
        const auto lg = so3_log<OpsF32, float>(Rerr);
#pragma unroll
        for (int i = 0; i < 9; ++i) S.G[c][i] = G[i];
        S.x[c][0] = xpt.x;
        S.x[c][1] = xpt.y;
        S.x[c][2] = xpt.z;
        S.phi[c][0] = lg.phi.x;
        S.phi[c][1] = lg.phi.y;
        S.phi[c][2] = lg.phi.z;
        S.beta[c] = jl_inv_beta<float>(lg.theta, lg.s, lg.c);
        S.F[r0] = t.x;
        S.F[r0 + 1] = t.y;
        S.F[r0 + 2] = t.z;
        S.F[r0 + 3] = lg.phi.x;
        S.F[r0 + 4] = lg.phi.y;
        S.F[r0 + 5] = lg.phi.z;
      }
    }
  });
  __syncwarp();
  const float fv = lane < K ? S.F[lane] : 0.f;
  if constexpr (MODE < 0) {
    const float r2 = warp_sum(fv * fv);
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
    if constexpr (MODE == WI_CHECK) return false;
  }
  // 5. Jacobian columns, joint j on lane j (a constraint without a column in
  // the slot's joints only writes its zeros)
  static_for<SL>([&](auto SS) {
    constexpr int s = decltype(SS)::value;
    const int j = lane + 32 * s;
    if (j < D) {
      const bool rev = tb.rev[j] != 0;
      const V3<float> z{S.T[j][2], S.T[j][6], S.T[j][10]};
      const V3<float> o{S.T[j][3], S.T[j][7], S.T[j][11]};
      static_for<P::NC>([&](auto CC) {
        constexpr int c = decltype(CC)::value;
        constexpr int kind = P::ckind(c);
        constexpr int r0 = roff<P>(c);
        const float sg = tb.coef[c][j];
        if constexpr ((MODE >= 0 && c != MODE) || !any_column<P>(c, 32 * s, 32 * s + 32)) {
#pragma unroll
          for (int r = 0; r < cdim(kind); ++r) S.J[j][r0 + r] = 0.f;
        } else if constexpr (kind == K_AXIS) {
          const V3<float> d = cross(z, V3<float>{S.za[c][0], S.za[c][1], S.za[c][2]});
          S.J[j][r0] = rev ? sg * d.x : 0.f;
          S.J[j][r0 + 1] = rev ? sg * d.y : 0.f;
        } else if constexpr (kind == K_COM || kind == K_HULL) {
          const float Mj = tb.msub[j];
          const V3<float> r{fmaf(-Mj, o.x, S.C[j][0]), fmaf(-Mj, o.y, S.C[j][1]), fmaf(-Mj, o.z, S.C[j][2])};
          const V3<float> d = cross(z, r);
          const float fpr = Mj * m.inv_mass;
          float g0 = sg * (rev ? d.x * m.inv_mass : fpr * z.x);
          float g1 = sg * (rev ? d.y * m.inv_mass : fpr * z.y);
          if constexpr (kind == K_HULL) {  // inside: 0; on an edge: n n^T g; at a vertex: g
            const int hm = S.hmode[c];
            if (hm == 0) {
              g0 = g1 = 0.f;
            } else if (hm == 1) {
              const float sd = fmaf(S.hn[c][0], g0, S.hn[c][1] * g1);
              g0 = S.hn[c][0] * sd;
              g1 = S.hn[c][1] * sd;
            }
          }
          S.J[j][r0] = g0;
          S.J[j][r0 + 1] = g1;
        } else {
          float G[9];
#pragma unroll
          for (int i = 0; i < 9; ++i) G[i] = S.G[c][i];
          const V3<float> xp{S.x[c][0], S.x[c][1], S.x[c][2]};
          const V3<float> v = rev ? cross(z, sub(xp, o)) : z;
          const V3<float> vt = mulv(G, v);
          S.J[j][r0] = sg * vt.x;
          S.J[j][r0 + 1] = sg * vt.y;
          S.J[j][r0 + 2] = sg * vt.z;
          const V3<float> w = jl_inv_apply(V3<float>{S.phi[c][0], S.phi[c][1], S.phi[c][2]}, S.beta[c], mulv(G, z));
          S.J[j][r0 + 3] = rev ? sg * w.x : 0.f;
          S.J[j][r0 + 4] = rev ? sg * w.y : 0.f;
          S.J[j][r0 + 5] = rev ? sg * w.z : 0.f;
        }
      });
    }
  });
  __syncwarp();
  // 6. Gram row `lane`: acc[b] = sum_j J[j][lane] J[j][b] (+ lambda on the diagonal)
  float acc[KP];
#pragma unroll
  for (int b = 0; b < KP; ++b) acc[b] = 0.f;
  const int arow = lane < K ? lane : 0;
  // per run of joints with the same row groups: only the groups holding a
  // structural nonzero of those columns are read and accumulated
  constexpr GramRuns<P> GR = gram_runs<P>();
  static_for<GR.n>([&](auto RR) {
    constexpr int rn = decltype(RR)::value;
    constexpr unsigned msk = GR.mask[rn];
    if constexpr (msk != 0u) {
#pragma unroll 1
      for (int j = GR.begin[rn]; j < GR.begin[rn + 1]; ++j) {
        const float ja = S.J[j][arow];
        const float4 *row = reinterpret_cast<const float4 *>(S.J[j]);
        static_for<KP / 4>([&](auto BB) {
          constexpr int b4 = decltype(BB)::value;
          if constexpr ((msk >> b4) & 1u) {
            const float4 v = row[b4];
            acc[4 * b4] = fmaf(ja, v.x, acc[4 * b4]);
            acc[4 * b4 + 1] = fmaf(ja, v.y, acc[4 * b4 + 1]);
            acc[4 * b4 + 2] = fmaf(ja, v.z, acc[4 * b4 + 2]);
            acc[4 * b4 + 3] = fmaf(ja, v.w, acc[4 * b4 + 3]);
          }
        });
      }
    }
  });
  float diag = a.lambda;
  if constexpr (MODE >= 0) {  // masked rows: unit diagonal, zero right-hand side
    constexpr int lo = roff<P>(MODE), hi = roff<P>(MODE) + cdim(P::ckind(MODE));
    if (lane < lo || lane >= hi) diag = 1.f;
  }
#pragma unroll
  for (int b = 0; b < K; ++b)
    if (b == lane) acc[b] += diag;
  // 7. Cholesky, row `lane` in registers; column k exchanged through shared memory
  float minpiv = FLT_MAX;
  float inv_diag = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float piv = __shfl_sync(FULL, acc[k], k);
    minpiv = fminf(minpiv, piv);
    const float ik = rsqrtf(piv);
    if (lane == k) inv_diag = ik;
    const float lik = (lane == k) ? piv * ik : acc[k] * ik;
    if (lane >= k) acc[k] = lik;
    if (lane < K) S.y[lane] = lik;
    __syncwarp();
    if (lane > k && lane < K) {
#pragma unroll
      for (int b = k + 1; b < K; ++b) acc[b] = fmaf(-lik, S.y[b], acc[b]);
    }
    __syncwarp();
  }
  if (!(minpiv >= a.pivot)) {  // includes NaN: this configuration continues in FP64
    fl |= FL_INT_NEEDS_F64;
    return true;
  }
  if (lane < K) {
#pragma unroll
    for (int b = 0; b < K; ++b) S.L[lane][b] = acc[b];
  }
  // (L L^T)^{-1} b with row i of L in lane i's registers and L in shared memory:
  // forward substitution broadcasts y_k, back substitution reads L[i][lane]
  auto subst = [&](float tv) -> float {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float yk = __shfl_sync(FULL, tv * inv_diag, k);
      if (lane == k) tv = yk;
      if (lane > k) tv = fmaf(-acc[k], yk, tv);
    }
    __syncwarp();
#pragma unroll
    for (int i = K - 1; i >= 0; --i) {
      const float zi = __shfl_sync(FULL, tv * inv_diag, i);
      if (lane == i) tv = zi;
      if (lane < i) tv = fmaf(-S.L[i][lane], zi, tv);
    }
    return tv;
  };
  // dq = J^T y for the y held by lanes < K (joint j on lane j)
  float dq[SL];
  auto jt_y = [&](float yv) {
    if (lane < K) S.y[lane] = yv;
    __syncwarp();
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int j = lane + 32 * s;
      dq[s] = 0.f;
      if (j < D) {
        float acc2 = 0.f;
#pragma unroll
        for (int b = 0; b < K; ++b) acc2 = fmaf(S.J[j][b], S.y[b], acc2);
        dq[s] = acc2;
        S.dq[j] = acc2;
      }
    }
    __syncwarp();
  };
  float yv = subst(fv);
  jt_y(yv);
  // one refinement step with the residual from J (corrected semi-normal equations):
  // r = F - J (J^T y) - lambda y
  float rv = 0.f;
  if (lane < K) {
    float jd = 0.f;
#pragma unroll 4
    for (int j = 0; j < D; ++j) jd = fmaf(S.J[j][lane], S.dq[j], jd);
    rv = fmaf(-a.lambda, yv, fv - jd);
  }
  __syncwarp();
  yv += subst(rv);
  jt_y(yv);
#pragma unroll
  for (int s = 0; s < SL; ++s) dq[s] *= a.alpha;
  if constexpr (MODE >= 0) {  // a sub-step of a sweep: the sweep does the rest
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int j = lane + 32 * s;
      if (j < D) S.q[j] -= dq[s];
    }
    __syncwarp();
    return false;
  }
  float s2 = 0.f;
#pragma unroll
  for (int s = 0; s < SL; ++s) s2 = fmaf(dq[s], dq[s], s2);
  s2 = warp_sum(s2);
  if (a.max_step2 > 0.f && s2 > a.max_step2) {
    fl |= FL_DIV;
    return true;
  }
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int j = lane + 32 * s;
    if (j < D) S.q[j] -= dq[s];
  }
  ++it;
  fl &= ~FL_INT_FORCE;
  __syncwarp();
  if (!(s2 <= FLT_MAX)) {
    fl |= FL_NONFINITE;
    return true;
  }
  return false;
}

// One sweep of the cyclic form (Sec. IV-C) on the warp's configuration: the
// stopping test on the stacked F, then one masked LM step per constraint.
// MaxDistance applies to the sweep; a small pivot returns the configuration,
// at the start of its sweep, to the FP64 path.
template <class P, class A>
__device__ __forceinline__ bool warp_sweep(const A &a, const WarpTables<P> &tb, WarpState<P> &S, int &it,
                                           uint32_t &fl) {
  constexpr int D = P::D, SL = (D + 31) / 32;
  const int lane = threadIdx.x & 31;
  if (warp_iter<P, WI_CHECK>(a, tb, S, it, fl)) return true;
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int j = lane + 32 * s;
    if (j < D) S.q0[j] = S.q[j];
  }
  __syncwarp();
  bool left = false;
  static_for<P::NC>([&](auto CC) {
    if (!left) left = warp_iter<P, decltype(CC)::value>(a, tb, S, it, fl);
  });
  float s2 = 0.f;
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int j = lane + 32 * s;
    if (j < D) s2 = fmaf(S.q[j] - S.q0[j], S.q[j] - S.q0[j], s2);
  }
  s2 = warp_sum(s2);
  if (left || (a.max_step2 > 0.f && s2 > a.max_step2)) {
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int j = lane + 32 * s;
      if (j < D) S.q[j] = S.q0[j];
    }
    __syncwarp();
    if (!left) fl |= FL_DIV;
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

// 128 registers (4 blocks of 4 warps per SM): the extra spills sit in the rare
// FP64 paths; 16 resident warps instead of 12 measured 11 % faster.
template <class P, int W, bool CYC>
__global__ void __launch_bounds__(W * 32, 512 / (W * 32)) k_project_warp(const __grid_constant__ WarpArgs<P> a) {
  constexpr int D = P::D;
  constexpr int SL = (D + 31) / 32;
  __shared__ WarpTables<P> tb;
  __shared__ WarpState<P> ws[W];
  __shared__ long long s_item[W][32];
  __shared__ uint32_t s_meta[W][32];
  __shared__ long long s_ritem[W][RETRY_CAP];  // sent back to the FP32 loop by the acceptance
  __shared__ uint32_t s_rmeta[W][RETRY_CAP];
  {
    const int *src = reinterpret_cast<const int *>(&a.t);
    int *dst = reinterpret_cast<int *>(&tb);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(WarpTables<P>) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  WarpState<P> &S = ws[wib];
  long long qn = 0, qe = 0;
  bool more = true;
  int pend = 0;
  int nret = 0;  // configurations to retry in FP32 after a failed acceptance
  while (true) {
    // a configuration to retry first, else the next one (chunks of `chunk` per atomic)
    const bool from_retry = nret > 0;
    if (!from_retry && qn >= qe && more) {
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(a.counter, static_cast<unsigned long long>(a.chunk));
      b = __shfl_sync(FULL, b, 0);
      if (static_cast<long long>(b) >= a.total) {
        more = false;
      } else {
        qn = static_cast<long long>(b);
        qe = qn + a.chunk < a.total ? qn + a.chunk : a.total;
      }
    }
    const bool have = from_retry || qn < qe;
    if (have) {
      long long item;
      int it = 0;
      uint32_t fl = 0;
      if (from_retry) {  // one more FP32 step from the parked iterate
        --nret;
        item = s_ritem[wib][nret];
        const uint32_t meta = s_rmeta[wib][nret];
        it = static_cast<int>(meta & 0xffu);
        fl = ((meta >> 8) & ~(FL_INT_FP32CONV | FL_INT_NEEDS_F64)) | FL_INT_FORCE;
#pragma unroll
        for (int s = 0; s < SL; ++s) {
          const int j = lane + 32 * s;
          if (j < D) S.q[j] = MCP_CHK(item, a.ld_out) ? a.q_out[j * a.ld_out + item] : 0.f;
        }
      } else {
        item = qn++;
#pragma unroll
        for (int s = 0; s < SL; ++s) {
          const int j = lane + 32 * s;
          if (j < D) S.q[j] = MCP_CHK(item, a.src.ld) ? a.src.q[j * a.src.ld + item] : 0.f;
        }
      }
      __syncwarp();
      if constexpr (CYC) {
        while (!warp_sweep<P>(a, tb, S, it, fl)) {
        }
      } else {
        while (!warp_iter<P, WI_STACKED>(a, tb, S, it, fl)) {
        }
      }
#pragma unroll
      for (int s = 0; s < SL; ++s) {
        const int j = lane + 32 * s;
        if (j < D && MCP_CHK(item, a.ld_out)) a.q_out[j * a.ld_out + item] = S.q[j];
      }
      if (lane == 0) {
        s_item[wib][pend] = item;
        s_meta[wib][pend] = static_cast<uint32_t>(it) | (fl << 8);
      }
      ++pend;
      __syncwarp();
    }
    const bool drained = !have && !more;  // (no retry pending either)
    if (pend == 32 || (drained && pend > 0)) {
      const bool room = nret + pend <= RETRY_CAP;
      bool retry = false;
      long long it_item = 0;
      uint32_t meta = 0;
      if (lane < pend) {
        meta = s_meta[wib][lane];
        it_item = s_item[wib][lane];
        retry = accept_one<P, CYC ? FORM_CYCLIC : FORM_STACKED>(a, it_item, static_cast<int>(meta & 0xffu),
                                                                meta >> 8, room);
      }
      const unsigned rm = __ballot_sync(FULL, retry);
      __syncwarp();
      if (retry) {
        const int rp = nret + __popc(rm & ((1u << lane) - 1u));
        s_ritem[wib][rp] = it_item;
        s_rmeta[wib][rp] = meta;
      }
      nret += __popc(rm);
      pend = 0;
      __syncwarp();
    }
    if (drained && nret == 0) break;
  }
}

template <class P>
WarpTables<P> make_warp_tables(const ModelT<float> &m) {
  static_assert(dfs_preorder<P>(), "warp kernel needs joints in depth-first order");
  WarpTables<P> t{};
  for (int j = 0; j < P::D; ++j) {
    for (int e = 0; e < 12; ++e) t.X[j][e] = m.X[j][e];
    t.mass[j] = m.mass[j];
    for (int r = 0; r < 3; ++r) t.com[j][r] = m.com[j][r];
    t.com[j][3] = 0.f;
    t.msub[j] = m.msub[j];
    t.parent[j] = P::parent(j);
    t.rev[j] = P::jtype(j) == REV ? 1 : 0;
    int end = j + 1;
    while (end < P::D && is_anc<P>(j, end)) ++end;
    t.sub_end[j] = end;
    for (int c = 0; c < P::NC; ++c) t.coef[c][j] = static_cast<float>(col_sign<P>(c, j));
  }
  for (int f = 0; f < P::NF; ++f)
    for (int e = 0; e < 12; ++e) t.fX[f][e] = m.fX[f][e];
  return t;
}

template <class P>
cudaError_t launch_project_warp(const HostModel &hm, const ProjCall &c, int *launches) {
  if (c.total <= 0) return cudaSuccess;
  if (c.precision == 1 || c.segments) return cudaErrorNotSupported;
  cudaError_t err = cudaMemsetAsync(c.counter, 0, sizeof(unsigned long long), c.stream);
  if (err != cudaSuccess) return err;
  constexpr int W = 4;
  WarpArgs<P> a;
  a.m = hm.m32;
  a.t = make_warp_tables<P>(hm.m32);
  a.m64 = hm.d_m64;
  a.tab = hm.d_tab;
  a.src = BatchSrc<float>{static_cast<const float *>(c.q_in), c.ld_in};
  a.q_out = static_cast<float *>(c.q_out);
  a.ld_out = c.ld_out;
  a.flags = c.flags;
  a.iters = c.iters;
  a.resid = c.resid;
  a.counter = c.counter;
  a.total = c.total;
  a.chunk = 8;
  a.cap = c.cap;
  a.tol2 = static_cast<float>(c.tol * c.tol);
  a.lambda = static_cast<float>(c.lambda);
  a.max_step2 = c.max_step > 0 ? static_cast<float>(c.max_step * c.max_step) : 0.f;
  a.pivot = static_cast<float>(c.pivot);
  a.tol2_64 = c.tol * c.tol;
  a.lambda64 = c.lambda;
  a.alpha = static_cast<float>(c.alpha);
  if (c.outer) return cudaErrorNotSupported;
  auto go = [&](auto kern) -> cudaError_t {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, 0);
    if (per_sm < 1) per_sm = 1;
    long long blocks = static_cast<long long>(hm.sm_count) * per_sm;
    const long long need = (c.total + a.chunk * W - 1) / (a.chunk * W);
    if (blocks > need) blocks = need;
    kern<<<static_cast<unsigned>(blocks), W * 32, 0, c.stream>>>(a);
    *launches += 1;
    return cudaGetLastError();
  };
  if (c.cyclic && P::NC > 1) return go(k_project_warp<P, W, true>);
  return go(k_project_warp<P, W, false>);
}

}  // namespace mcp
