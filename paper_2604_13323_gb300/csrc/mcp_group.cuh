// Group-cooperative projection for large tree problems (the 36-DoF humanoid
// with 20 stacked equations): four lanes share one configuration, so a warp
// advances eight configurations at once.  One warp per configuration (the
// warp kernel) leaves most lanes idle in every sequential stage (a 20-step
// Cholesky, the substitutions, rows 20..31 of the Gram build); four lanes
// keep the per-configuration work almost as dense as one thread would, while
// the configuration's Jacobian, Gram matrix and factor live in shared memory
// instead of one thread's registers.
//
// Per FP32 iteration of Alg. 2 (stacked F, inner LM form), for each group of
// four lanes and its configuration:
//   1. FK along the kinematic tree: every lane walks the joints of the chains
//      it owns (limbs, assigned by longest-first scheduling) and the shared
//      trunk (computed by every lane), storing the joint axes and origins and
//      the mass moments m_j c_j; a prismatic chain at the root (the floating
//      base's translations) is placed in closed form, its rotations being
//      constant;
//   2. subtree mass moments C_j = m_j c_j + sum over children, limbs first,
//      then the trunk;
//   3. residuals, constraint c on lane c mod 4 (the pose and relative-pose
//      constraints on one code path, so that their lanes run it together);
//      ||F|| by a group reduction;
//   4. the structural nonzeros of J, as (joint, constraint) segments spread
//      over the lanes;
//   5. the Gram matrix J J^T by blocks: each lane accumulates whole row-block
//      pairs (6x6, 2x6, 2x2) over the joints both blocks share, in registers;
//   6. Cholesky with rows i = 4m + g on lane g (registers), column k of L
//      exchanged through shared memory (which keeps L by columns for the
//      back substitution); blocks of L that the symbolic factorisation
//      proves zero (feet rows against hand columns) are skipped at compile
//      time, in the factorisation and both substitutions;
//   7. forward / back substitution, dq = J^T y, one refinement step
//      (r = F - J dq - lambda y), alpha, MaxDistance, q <- q - dq.
// Finished configurations are parked and accepted in FP64 32 at a time, one
// per lane (the thread-level acceptance of the other kernels).
#pragma once

#include <algorithm>
#include <vector>

#include "mcp_warp.cuh"

namespace mcp {

// Limits of the work plan (the plan is copied into every block's shared
// memory, so they are kept near what the humanoid classes need).
constexpr int GG = 4;            // lanes per configuration
constexpr int GCPW = 32 / GG;    // configurations per warp
constexpr int GMAX_FK = 20;      // FK steps per lane
constexpr int GMAX_CB = 16;      // own joints per lane (subtree moments)
constexpr int GMAX_CR = 16;      // trunk joints
constexpr int GMAX_CH = 4;       // children per joint
constexpr int GMAX_JI = 16;      // Jacobian segments per lane and segment size
constexpr int GMAX_DQ = 20;      // dq joints per lane
constexpr int GMAX_T = 2;        // Gram / refinement tasks per lane and phase
constexpr int GMAX_POOL = 192;   // joint lists of the tasks
constexpr int GMAX_PRE = 3;      // prismatic root joints placed in closed form

template <class P>
__host__ __device__ constexpr bool grp_pose_like(int c) {
  return P::ckind(c) == K_POSE || P::ckind(c) == K_REL;
}
template <class P>
__host__ __device__ constexpr bool grp_com_like(int c) {
  return P::ckind(c) == K_COM || P::ckind(c) == K_HULL;
}
template <class P>
__host__ __device__ constexpr bool grp_supported() {
  for (int c = 0; c < P::NC; ++c)
    if (!grp_pose_like<P>(c) && !grp_com_like<P>(c)) return false;
  return P::D <= 64 && kdim<P>() <= 4 * 5 && dfs_preorder<P>();
}
// Per-constraint data slots: the pose-like constraints (error frame G, point
// x, log-map vector) and the support-hull ones (nearest-edge data) are stored
// per kind, not per constraint, so that the shared state holds no unused rows.
template <class P>
__host__ __device__ constexpr int grp_pslot(int c) {
  int n = 0;
  for (int b = 0; b < c; ++b) n += grp_pose_like<P>(b) ? 1 : 0;
  return n;
}
template <class P>
__host__ __device__ constexpr int grp_hslot(int c) {
  int n = 0;
  for (int b = 0; b < c; ++b) n += P::ckind(b) == K_HULL ? 1 : 0;
  return n;
}
template <class P>
__host__ __device__ constexpr int grp_npose() { return grp_pslot<P>(P::NC); }
template <class P>
__host__ __device__ constexpr int grp_nhull() { return grp_hslot<P>(P::NC); }

// Jacobian segments: (joint j, constraint c) with a structural nonzero, j-major
template <class P>
__host__ __device__ constexpr int grp_nseg_floats() {
  int n = 0;
  for (int j = 0; j < P::D; ++j)
    for (int c = 0; c < P::NC; ++c)
      if (col_sign<P>(c, j) != 0) n += cdim(P::ckind(c));
  return n;
}
// Floats of the 2-row (CoM-like) segments, which come first in the Jacobian's
// space; the subtree moments C_j (3 floats per joint) are kept right after
// them, where the 6-row segments are written once the 2-row ones are built.
template <class P>
__host__ __device__ constexpr int grp_cbase() {
  int n = 0;
  for (int j = 0; j < P::D; ++j)
    for (int c = 0; c < P::NC; ++c)
      if (col_sign<P>(c, j) != 0 && grp_com_like<P>(c)) n += cdim(P::ckind(c));
  return (n + 3) & ~3;
}

// L by columns, packed: rows k .. K-1 of column k from lcol_base(k)
template <int K>
__host__ __device__ constexpr int lcol_base(int k) {
  int o = 0;
  for (int t = 0; t < k; ++t) o += K - t;
  return o;
}

// Structural nonzeros of the Cholesky factor of A = J J^T + lambda I, row by
// row (bit b of row i: L[i][b] may be nonzero).  The symbolic factorisation:
// L[i][b] is nonzero where A[i][b] is (rows i and b of J share a joint) or
// where L[i][j] and L[b][j] are both nonzero for some column j < b.
template <class P>
__host__ __device__ constexpr uint32_t l_row_pattern(int row) {
  constexpr int K = kdim<P>();
  uint64_t jm[MAXK] = {};  // joints of row i of J
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < P::D; ++j)
      if (jnz<P>(i, j)) jm[i] |= uint64_t(1) << j;
  uint32_t nz[MAXK] = {};
  for (int i = 0; i < K; ++i)
    for (int b = 0; b <= i; ++b) {
      bool v = (b == i) || (jm[i] & jm[b]) != 0;
      for (int j = 0; j < b && !v; ++j) v = ((nz[i] >> j) & 1u) != 0 && ((nz[b] >> j) & 1u) != 0;
      if (v) nz[i] |= 1u << b;
    }
  return nz[row];
}
template <class P, int I>
struct LRow {
  static constexpr uint32_t value = l_row_pattern<P>(I);
};
// Rows 4 mm .. 4 mm + 3 (one per lane of a group) all lie below row k and
// are structurally zero in column k of L: the group skips their update.
template <class P, int MM, int KC>
__host__ __device__ constexpr bool l_col_block_zero() {
  constexpr uint32_t m = LRow<P, GG * MM>::value | LRow<P, GG * MM + 1>::value | LRow<P, GG * MM + 2>::value |
                         LRow<P, GG * MM + 3>::value;
  return GG * MM > KC && ((m >> KC) & 1u) == 0u;
}
// Columns 4 mm .. 4 mm + 3 all lie left of column k and row k of L is
// structurally zero in them.
template <class P, int KR, int MM>
__host__ __device__ constexpr bool l_row_seg_zero() {
  return GG * MM + GG - 1 < KR && ((LRow<P, KR>::value >> (GG * MM)) & 0xFu) == 0u;
}

// Tasks of the Gram build and of the refinement residual: row blocks (a, b)
// (b unused for the refinement) and a joint list pool[off, off + n).
struct GrpTask {
  int8_t a, b, n, pad;
  int16_t off, pad2;
};

template <class P>
struct GroupPlan {
  static constexpr int D = P::D, NC = P::NC;
  // 1. FK: per lane and step the joint, the parent source (0: the previous
  // step, 1 / 2: saved slot 0 / 1, 3: the world), the slot to save into and
  // whether this lane writes the joint's data
  int8_t fk_j[GG][GMAX_FK];
  int8_t fk_par[GG][GMAX_FK];
  int8_t fk_save[GG][GMAX_FK];
  int8_t fk_store[GG][GMAX_FK];
  // 2. subtree moments: own joints (reverse preorder) per lane, then the trunk
  int8_t cb_j[GG][GMAX_CB];
  int8_t cr_j[GMAX_CR];
  int8_t child[D][GMAX_CH];
  int8_t roots[4];
  // 4. Jacobian segments per lane: 6-row and 2-row
  int8_t j6_j[GG][GMAX_JI], j6_c[GG][GMAX_JI];
  int8_t j2_j[GG][GMAX_JI], j2_c[GG][GMAX_JI];
  // 7. dq joints per lane (every joint on exactly one lane)
  int8_t dq_j[GG][GMAX_DQ];
  int16_t joff[NC][D];  // segment offset of (j, c), -1: structural zero
  int8_t croff[NC];     // first row of constraint c
  int16_t lcol[GG * 5];  // start of column i of L (shared memory, by columns)
  uint32_t amask[GG * 5];  // row i of J J^T: bit b set if rows i and b share a joint
                           // (the other entries are never written: structural zeros)
  int8_t chull[NC];     // constraint c is the support-hull kind
  int8_t pslot[NC];     // slot of constraint c among the pose-like ones (-1: other kinds)
  int8_t hslot[NC];     // slot of constraint c among the support-hull ones (-1: other kinds)
  int8_t crel[NC];      // pose-like constraint c is the relative pose of two frames
  int8_t cfa[NC], cfb[NC];  // its frames (cfb: the relative pose's second frame, else cfa)
  // 5. Gram phases (6x6, 6x2, 2x6, 2x2 row-block pairs) and 7. refinement
  // phases (6-row, 2-row blocks): tasks per lane.  The diagonal blocks and
  // refinement rows of 2-row constraints (the CoM, over every joint) are
  // summed over the dq partition instead, four lanes and a group reduction.
  GrpTask gt[4][GG][GMAX_T];
  GrpTask rt[2][GG][GMAX_T];
  int8_t pool[GMAX_POOL];
  int n_fk, n_cb, n_cr, n_roots, n_j6, n_j2, n_dq;
  int n_pre;  // leading FK steps of every lane placed in closed form (a prismatic root chain)
  int g_nt[4], g_len[4][GMAX_T];  // per phase: task slots, longest list per slot
  int r_nt[2], r_len[2][GMAX_T];
};

// Host: the plan of problem class P.  Returns false (with the reason) when
// the tree or the constraint stack does not fit the plan's limits.
template <class P>
bool make_group_plan(GroupPlan<P> &pl, const char **why) {
  constexpr int D = P::D, NC = P::NC;
  pl = GroupPlan<P>{};
  auto fail = [&](const char *w) {
    if (why) *why = w;
    return false;
  };
  std::vector<std::vector<int>> ch(D);
  for (int j = 0; j < D; ++j)
    if (P::parent(j) >= 0) ch[P::parent(j)].push_back(j);
  // chains: maximal paths whose inner joints have exactly one child
  std::vector<std::vector<int>> chains;
  std::vector<int> chain_of(D, -1);
  for (int j = 0; j < D; ++j) {
    if (!(P::parent(j) < 0 || ch[P::parent(j)].size() != 1)) continue;
    std::vector<int> c{j};
    while (ch[c.back()].size() == 1) c.push_back(ch[c.back()][0]);
    for (int v : c) chain_of[v] = static_cast<int>(chains.size());
    chains.push_back(c);
  }
  const int nch = static_cast<int>(chains.size());
  // leaf chains to lanes, longest first, onto the least loaded lane
  std::vector<int> owner_c(nch, -2), load(GG, 0), leaves;
  for (int c = 0; c < nch; ++c)
    if (ch[chains[c].back()].empty()) leaves.push_back(c);
  std::stable_sort(leaves.begin(), leaves.end(),
                   [&](int x, int y) { return chains[x].size() > chains[y].size(); });
  for (int c : leaves) {
    const int g = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
    owner_c[c] = g;
    load[g] += static_cast<int>(chains[c].size());
  }
  // inner chains: the lane of all their descendants, else every lane (-1);
  // in preorder a chain's descendants start after it
  for (int c = nch - 1; c >= 0; --c) {
    if (owner_c[c] != -2) continue;
    int o = -2;
    for (int k : ch[chains[c].back()]) {
      const int oc = owner_c[chain_of[k]];
      o = (o == -2) ? oc : (o == oc ? o : -1);
    }
    owner_c[c] = o;
  }
  std::vector<int> owner(D);
  for (int j = 0; j < D; ++j) owner[j] = owner_c[chain_of[j]];
  // 1. FK schedules
  int n_fk = 0;
  for (int g = 0; g < GG; ++g) {
    std::vector<int> js;
    for (int j = 0; j < D; ++j)
      if (owner[j] == g || owner[j] == -1) js.push_back(j);
    if (static_cast<int>(js.size()) > GMAX_FK) return fail("FK schedule too long");
    std::vector<int> slot_of(D, -1);
    int nslot = 0;
    // a parent that is not the previous step must have been saved
    for (size_t k = 0; k < js.size(); ++k) {
      const int p = P::parent(js[k]);
      if (p >= 0 && !(k > 0 && js[k - 1] == p) && slot_of[p] < 0) {
        if (nslot >= 2) return fail("more than two saved FK transforms");
        slot_of[p] = nslot++;
      }
    }
    for (int k = 0; k < GMAX_FK; ++k) {
      pl.fk_j[g][k] = -1;
      pl.fk_par[g][k] = 0;
      pl.fk_save[g][k] = -1;
      pl.fk_store[g][k] = 0;
    }
    for (size_t k = 0; k < js.size(); ++k) {
      const int j = js[k], p = P::parent(j);
      pl.fk_j[g][k] = static_cast<int8_t>(j);
      pl.fk_par[g][k] = static_cast<int8_t>(p < 0 ? 3 : ((k > 0 && js[k - 1] == p) ? 0 : 1 + slot_of[p]));
      pl.fk_save[g][k] = static_cast<int8_t>(slot_of[j]);
      pl.fk_store[g][k] = static_cast<int8_t>(owner[j] == g || (owner[j] == -1 && g == 0));
    }
    n_fk = std::max(n_fk, static_cast<int>(js.size()));
  }
  pl.n_fk = n_fk;
  // prismatic root prefix: joints 0 .. n_pre-1, prismatic, each the child of
  // the one before, at the head of every lane's schedule, with no transform
  // saved and no task frame among them
  {
    int n = 0;
    while (n < GMAX_PRE && n < D && P::jtype(n) == PRIS && P::parent(n) == n - 1) ++n;
    for (int f = 0; f < P::NF; ++f) n = std::min(n, P::frame_link(f) < n ? P::frame_link(f) : n);
    for (int g = 0; g < GG; ++g)
      for (int k = 0; k < n; ++k)
        if (pl.fk_j[g][k] != k || pl.fk_save[g][k] >= 0) n = k;
    for (int g = 0; g < GG; ++g)
      if (n > 0 && pl.fk_j[g][n] >= 0 && pl.fk_par[g][n] != 0) n = 0;
    pl.n_pre = n;
  }
  // 2. subtree moments
  int n_cb = 0;
  for (int g = 0; g < GG; ++g) {
    int n = 0;
    for (int k = 0; k < GMAX_CB; ++k) pl.cb_j[g][k] = -1;
    for (int j = D - 1; j >= 0; --j)
      if (owner[j] == g) {
        if (n >= GMAX_CB) return fail("too many joints on one lane");
        pl.cb_j[g][n++] = static_cast<int8_t>(j);
      }
    n_cb = std::max(n_cb, n);
  }
  pl.n_cb = n_cb;
  int n_cr = 0, n_roots = 0;
  for (int k = 0; k < GMAX_CR; ++k) pl.cr_j[k] = -1;
  for (int j = D - 1; j >= 0; --j)
    if (owner[j] == -1) {
      if (n_cr >= GMAX_CR) return fail("trunk too long");
      pl.cr_j[n_cr++] = static_cast<int8_t>(j);
    }
  pl.n_cr = n_cr;
  for (int j = 0; j < D; ++j) {
    if (static_cast<int>(ch[j].size()) > GMAX_CH) return fail("too many children");
    for (int k = 0; k < GMAX_CH; ++k)
      pl.child[j][k] = static_cast<int8_t>(k < static_cast<int>(ch[j].size()) ? ch[j][k] : -1);
    if (P::parent(j) < 0) {
      if (n_roots >= 4) return fail("too many roots");
      pl.roots[n_roots++] = static_cast<int8_t>(j);
    }
  }
  pl.n_roots = n_roots;
  // segment offsets (every segment size is even: float2 loads): the 2-row
  // segments of the CoM-like constraints first, then the 6-row ones, so that
  // the subtree moments can live where the 6-row segments go until the 2-row
  // segments are built from them (grp_cbase)
  int off = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int j = 0; j < D; ++j)
      for (int c = 0; c < NC; ++c) {
        if (pass == 0) pl.joff[c][j] = -1;
        if (col_sign<P>(c, j) != 0 && grp_com_like<P>(c) == (pass == 0)) {
          pl.joff[c][j] = static_cast<int16_t>(off);
          off += cdim(P::ckind(c));
        }
      }
  for (int i = 0; i < GG * 5; ++i) {
    pl.lcol[i] = static_cast<int16_t>(i < kdim<P>() ? lcol_base<kdim<P>()>(i) : 0);
    pl.amask[i] = 0u;
    for (int b = 0; b < kdim<P>() && i < kdim<P>(); ++b)
      for (int j = 0; j < D; ++j)
        if (jnz<P>(i, j) && jnz<P>(b, j)) pl.amask[i] |= 1u << b;
  }
  for (int c = 0; c < NC; ++c) {
    pl.croff[c] = static_cast<int8_t>(roff<P>(c));
    pl.chull[c] = static_cast<int8_t>(P::ckind(c) == K_HULL);
    pl.pslot[c] = static_cast<int8_t>(grp_pose_like<P>(c) ? grp_pslot<P>(c) : -1);
    pl.hslot[c] = static_cast<int8_t>(P::ckind(c) == K_HULL ? grp_hslot<P>(c) : -1);
    pl.crel[c] = static_cast<int8_t>(P::ckind(c) == K_REL);
    pl.cfa[c] = static_cast<int8_t>(grp_pose_like<P>(c) ? P::cfa(c) : 0);
    pl.cfb[c] = static_cast<int8_t>(P::ckind(c) == K_REL ? P::cfb(c) : pl.cfa[c]);
  }
  // 4. segments: a limb's segments on its lane, the trunk's on the lane with
  // the fewest segments of that size
  {
    int n6[GG] = {0, 0, 0, 0}, n2[GG] = {0, 0, 0, 0};
    for (int g = 0; g < GG; ++g)
      for (int k = 0; k < GMAX_JI; ++k) pl.j6_j[g][k] = pl.j6_c[g][k] = pl.j2_j[g][k] = pl.j2_c[g][k] = -1;
    for (int pass = 0; pass < 2; ++pass)  // owned joints first, then the trunk
      for (int j = 0; j < D; ++j) {
        if ((owner[j] == -1) != (pass == 1)) continue;
        for (int c = 0; c < NC; ++c) {
          if (col_sign<P>(c, j) == 0) continue;
          const bool six = grp_pose_like<P>(c);
          int *cnt = six ? n6 : n2;
          int g = owner[j];
          if (g < 0) g = static_cast<int>(std::min_element(cnt, cnt + GG) - cnt);
          if (cnt[g] >= GMAX_JI) return fail("too many Jacobian segments on one lane");
          (six ? pl.j6_j : pl.j2_j)[g][cnt[g]] = static_cast<int8_t>(j);
          (six ? pl.j6_c : pl.j2_c)[g][cnt[g]] = static_cast<int8_t>(c);
          ++cnt[g];
        }
      }
    pl.n_j6 = *std::max_element(n6, n6 + GG);
    pl.n_j2 = *std::max_element(n2, n2 + GG);
  }
  // 7. dq joints
  {
    int nd[GG] = {0, 0, 0, 0};
    for (int g = 0; g < GG; ++g)
      for (int k = 0; k < GMAX_DQ; ++k) pl.dq_j[g][k] = -1;
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j < D; ++j) {
        if ((owner[j] == -1) != (pass == 1)) continue;
        int g = owner[j];
        if (g < 0) g = static_cast<int>(std::min_element(nd, nd + GG) - nd);
        if (nd[g] >= GMAX_DQ) return fail("too many dq joints on one lane");
        pl.dq_j[g][nd[g]++] = static_cast<int8_t>(j);
      }
    pl.n_dq = *std::max_element(nd, nd + GG);
  }
  // 5. Gram tasks: row-block pairs (a, b), rows of a at or below those of b,
  // sharing at least one joint; 7. refinement tasks: one per row block
  int pool_n = 0;
  auto add_list = [&](const std::vector<int> &js) -> int {
    if (pool_n + static_cast<int>(js.size()) > GMAX_POOL) return -1;
    const int o = pool_n;
    for (int j : js) pl.pool[pool_n++] = static_cast<int8_t>(j);
    return o;
  };
  auto schedule = [&](std::vector<std::pair<GrpTask, std::vector<int>>> &tasks, GrpTask (*dst)[GMAX_T],
                      int &nt, int *len) -> bool {
    std::stable_sort(tasks.begin(), tasks.end(),
                     [](const auto &x, const auto &y) { return x.second.size() > y.second.size(); });
    int cnt[GG] = {0, 0, 0, 0}, lo[GG] = {0, 0, 0, 0};
    for (int g = 0; g < GG; ++g)
      for (int t = 0; t < GMAX_T; ++t) dst[g][t] = GrpTask{-1, -1, 0, 0, 0, 0};
    for (auto &tk : tasks) {
      const int g = static_cast<int>(std::min_element(lo, lo + GG) - lo);
      if (cnt[g] >= GMAX_T || tk.second.size() > 127) return false;
      const int o = add_list(tk.second);
      if (o < 0) return false;
      GrpTask t = tk.first;
      t.n = static_cast<int8_t>(tk.second.size());
      t.off = static_cast<int16_t>(o);
      dst[g][cnt[g]++] = t;
      lo[g] += static_cast<int>(tk.second.size());
    }
    nt = *std::max_element(cnt, cnt + GG);
    for (int t = 0; t < GMAX_T; ++t) {
      len[t] = 0;
      for (int g = 0; g < GG; ++g) len[t] = std::max(len[t], static_cast<int>(dst[g][t].n));
    }
    return true;
  };
  for (int ph = 0; ph < 4; ++ph) {
    const bool a6 = ph < 2, b6 = (ph % 2) == 0;
    std::vector<std::pair<GrpTask, std::vector<int>>> tasks;
    for (int a = 0; a < NC; ++a)
      for (int b = 0; b < NC; ++b) {
        if (roff<P>(a) < roff<P>(b)) continue;
        if (grp_pose_like<P>(a) != a6 || grp_pose_like<P>(b) != b6) continue;
        if (a == b && grp_com_like<P>(a)) continue;  // summed over the dq partition instead
        std::vector<int> js;
        for (int j = 0; j < D; ++j)
          if (col_sign<P>(a, j) != 0 && col_sign<P>(b, j) != 0) js.push_back(j);
        if (!js.empty()) tasks.push_back({GrpTask{static_cast<int8_t>(a), static_cast<int8_t>(b), 0, 0, 0, 0}, js});
      }
    if (!schedule(tasks, pl.gt[ph], pl.g_nt[ph], pl.g_len[ph])) return fail("Gram tasks exceed the plan");
  }
  for (int ph = 0; ph < 2; ++ph) {
    std::vector<std::pair<GrpTask, std::vector<int>>> tasks;
    for (int a = 0; a < NC; ++a) {
      if (!grp_pose_like<P>(a) || ph == 1) continue;  // 2-row blocks: summed over the dq partition
      std::vector<int> js;
      for (int j = 0; j < D; ++j)
        if (col_sign<P>(a, j) != 0) js.push_back(j);
      tasks.push_back({GrpTask{static_cast<int8_t>(a), -1, 0, 0, 0, 0}, js});
    }
    if (!schedule(tasks, pl.rt[ph], pl.r_nt[ph], pl.r_len[ph])) return fail("refinement tasks exceed the plan");
  }
  return true;
}

// Per-configuration state in shared memory.
template <class P>
struct __align__(16) GrpState {
  static constexpr int D = P::D, K = kdim<P>(), KP = (K + 3) & ~3, NF = P::NF, NC = P::NC;
  static constexpr int DP = (D + 3) & ~3;
  static constexpr int NJ = (grp_nseg_floats<P>() + 3) & ~3;
  static constexpr int LC = lcol_base<K>(K);
  static constexpr int K2 = K * (K + 1) / 2;
  static constexpr int NPOSE = grp_npose<P>() > 0 ? grp_npose<P>() : 1;
  static constexpr int NHULL = grp_nhull<P>() > 0 ? grp_nhull<P>() : 1;
  struct Eval {           // FK and residual data, live until J is built
    float zo[D][6];       // joint axis z and origin o (world)
    float G[NPOSE][9];    // pose-like constraints: rotation into the error frame
    float x[NPOSE][4];    // reference point of the translational rows
    float phi[NPOSE][4];  // log-map vector and J_l^-1 coefficient (w)
    float hn[NHULL][2];   // support hull: normal of the nearest edge
    int hmode[NHULL];     // support hull: 0 inside, 1 edge, 2 vertex
  };
  struct Solve {         // after the Cholesky (the refinement's residual r overwrites F)
    float Lc[LC];        // L by columns (rows k..K-1 of column k at lcol_base(k))
    float y[KP];
    float dq[DP];
  };
  float q[DP];
  float F[KP];  // F, then the refinement's residual r = F - J dq - lambda y
  float J[NJ];  // Jacobian segments; before they are built, the task frames (NF x 12)
  union alignas(16) {
    Eval e;
    float A[K2];  // Gram (packed lower triangle, row-major), read into registers before
    Solve s;      // L's columns overwrite it (y and dq lie beyond A)
  } u;
  static_assert(NJ >= NF * 12, "task frames live in the Jacobian's space");
  static_assert(NF * 12 <= grp_cbase<P>() || !needs_com<P>(), "task frames must not overlap the subtree moments");
  static_assert(grp_cbase<P>() + 3 * D <= NJ || !needs_com<P>(), "subtree moments must fit the 6-row segments' space");
  // the subtree moments C_j (m_j c_j, then the sum over the subtree), in the
  // Jacobian's space until the 2-row segments are built
  __device__ __forceinline__ float *C(int j) { return J + grp_cbase<P>() + 3 * j; }
  static_assert(LC >= K2, "y and dq must not overlap the Gram matrix");
};

// Model data the group kernel reads with runtime joint indices (shared memory).
template <class P>
struct GrpTables {
  float X[P::D][12];
  float fX[P::NF][12];
  float com[P::D][3];
  float mass[P::D];
  float msub[P::D];
  int8_t rev[P::D];
  int8_t sgn[P::NC][P::D];  // column sign of joint j in constraint c
  // the prismatic root chain in closed form (for its first GMAX_PRE joints):
  // with q = 0 joint i's frame sits at pre_c[i] with rotation R_i; its axis
  // is pre_a[i] = R_i e_z, so its origin is pre_c[i] + sum_{k <= i} q_k pre_a[k];
  // pre_mc[i] = m_i R_i com_i; pre_R = the rotation after the last of them
  float pre_R[GMAX_PRE][9];
  float pre_a[GMAX_PRE][3];
  float pre_c[GMAX_PRE][3];
  float pre_mc[GMAX_PRE][3];
  int8_t pad[4 - (P::D * (P::NC + 1)) % 4];  // whole words
};
// Shared-memory stride between the states of consecutive configurations: an
// odd number of 16-byte units, so that the eight configurations of a warp
// start in eight different banks (with an even number the lanes of the eight
// groups reading the same field of their state collide in one bank, up to
// eight ways; measured: 43.7 ms instead of 32.3 ms on the full humanoid batch).
template <class P>
__host__ __device__ constexpr size_t grp_state_stride() {
  constexpr size_t u = (sizeof(GrpState<P>) + 15) / 16;
  return 16 * ((u % 2 == 0) ? u + 1 : u);
}

template <class P>
GrpTables<P> make_grp_tables(const ModelT<float> &m, const ModelT<double> &m64) {
  GrpTables<P> t{};
  {  // the prismatic root chain, in FP64 then rounded
    double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, c[3] = {0, 0, 0};
    for (int i = 0; i < GMAX_PRE && i < P::D && P::jtype(i) == PRIS && P::parent(i) == i - 1; ++i) {
      const double *X = m64.X[i];
      double Rn[9], cn[3];
      for (int r = 0; r < 3; ++r) {
        cn[r] = c[r] + R[r * 3] * X[3] + R[r * 3 + 1] * X[7] + R[r * 3 + 2] * X[11];
        for (int cc = 0; cc < 3; ++cc)
          Rn[r * 3 + cc] = R[r * 3] * X[cc] + R[r * 3 + 1] * X[4 + cc] + R[r * 3 + 2] * X[8 + cc];
      }
      for (int e = 0; e < 9; ++e) R[e] = Rn[e];
      for (int r = 0; r < 3; ++r) c[r] = cn[r];
      for (int e = 0; e < 9; ++e) t.pre_R[i][e] = static_cast<float>(R[e]);
      for (int r = 0; r < 3; ++r) {
        t.pre_a[i][r] = static_cast<float>(R[r * 3 + 2]);
        t.pre_c[i][r] = static_cast<float>(c[r]);
        t.pre_mc[i][r] = static_cast<float>(m64.mass[i] * (R[r * 3] * m64.com[i][0] + R[r * 3 + 1] * m64.com[i][1] +
                                                           R[r * 3 + 2] * m64.com[i][2]));
      }
    }
  }
  for (int j = 0; j < P::D; ++j) {
    for (int e = 0; e < 12; ++e) t.X[j][e] = m.X[j][e];
    for (int r = 0; r < 3; ++r) t.com[j][r] = m.com[j][r];
    t.mass[j] = m.mass[j];
    t.msub[j] = m.msub[j];
    t.rev[j] = P::jtype(j) == REV ? 1 : 0;
    for (int c = 0; c < P::NC; ++c) t.sgn[c][j] = static_cast<int8_t>(col_sign<P>(c, j));
  }
  for (int f = 0; f < P::NF; ++f)
    for (int e = 0; e < 12; ++e) t.fX[f][e] = m.fX[f][e];
  return t;
}

template <class P>
struct GroupArgs {
  ModelT<float> m;
  GrpTables<P> t;
  GroupPlan<P> pl;
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

template <class P>
struct GrpShared {
  GrpTables<P> tb;
  GroupPlan<P> pl;
};

// Sum over the four lanes of a group.
__device__ __forceinline__ float grp_sum(float v) {
  v += __shfl_xor_sync(FULL, v, 1);
  v += __shfl_xor_sync(FULL, v, 2);
  return v;
}

__device__ __forceinline__ float2 lds2(const float *p) { return *reinterpret_cast<const float2 *>(p); }

// Residual of constraint c (compile time) into S.F, with the data the
// Jacobian needs; returns this constraint's squared norm.
template <class P, int c>
__device__ __forceinline__ float grp_residual(const ModelT<float> &m, GrpState<P> &S, const float (&tot)[3]) {
  constexpr int kind = P::ckind(c);
  constexpr int r0 = roff<P>(c);
  auto &E = S.u.e;
  const float(*Tf)[12] = reinterpret_cast<const float(*)[12]>(S.J);
  if constexpr (kind == K_COM) {
    const float f0 = fmaf(tot[0], m.inv_mass, -m.ctgt[c][0]);
    const float f1 = fmaf(tot[1], m.inv_mass, -m.ctgt[c][1]);
    S.F[r0] = f0;
    S.F[r0 + 1] = f1;
    return fmaf(f0, f0, f1 * f1);
  } else if constexpr (kind == K_HULL) {
    const float cx = tot[0] * m.inv_mass, cy = tot[1] * m.inv_mass;
    float px, py, nx, ny;
    constexpr int hs = grp_hslot<P>(c);
    E.hmode[hs] = polygon_nearest<float>(m.cB[c], static_cast<int>(m.ctgt[c][0]), cx, cy, px, py, nx, ny);
    E.hn[hs][0] = nx;
    E.hn[hs][1] = ny;
    const float f0 = cx - px, f1 = cy - py;
    S.F[r0] = f0;
    S.F[r0 + 1] = f1;
    return fmaf(f0, f0, f1 * f1);
  } else {
    static_assert(kind == K_POSE || kind == K_REL, "pose-like constraint expected");
    constexpr int ps = grp_pslot<P>(c);
    float Pr[9], Rerr[9], G[9];
    load_R(m.cPinv[c], Pr);
    const V3<float> Pp = load_p(m.cPinv[c]);
    V3<float> t, xpt;
    constexpr int fa = P::cfa(c);
    float Ra[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) Ra[r * 3 + cc] = Tf[fa][r * 4 + cc];
    const V3<float> pa{Tf[fa][3], Tf[fa][7], Tf[fa][11]};
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
        for (int cc = 0; cc < 3; ++cc) Rb[r * 3 + cc] = Tf[fb][r * 4 + cc];
      const V3<float> pb{Tf[fb][3], Tf[fb][7], Tf[fb][11]};
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
    for (int i = 0; i < 9; ++i) E.G[ps][i] = G[i];
    E.x[ps][0] = xpt.x;
    E.x[ps][1] = xpt.y;
    E.x[ps][2] = xpt.z;
    E.phi[ps][0] = lg.phi.x;
    E.phi[ps][1] = lg.phi.y;
    E.phi[ps][2] = lg.phi.z;
    E.phi[ps][3] = jl_inv_beta<float>(lg.theta, lg.s, lg.c);
    S.F[r0] = t.x;
    S.F[r0 + 1] = t.y;
    S.F[r0 + 2] = t.z;
    S.F[r0 + 3] = lg.phi.x;
    S.F[r0 + 4] = lg.phi.y;
    S.F[r0 + 5] = lg.phi.z;
    return fmaf(t.x, t.x, fmaf(t.y, t.y, fmaf(t.z, t.z, fmaf(lg.phi.x, lg.phi.x, fmaf(lg.phi.y, lg.phi.y, lg.phi.z * lg.phi.z)))));
  }
}

// Residual of pose-like constraint c (run time: the pose and relative-pose
// constraints of a stack run one code path, on their lanes at once) into
// S.F, with the data the Jacobian needs; returns its squared norm.
//   pose (Eq. 1):          G = P^-1_R,          R_err = G (R_a Q^-1_R),
//                          x = p_a + R_a Q^-1_p, t = G x + P^-1_p;
//   relative pose (Eq. 2): G = P^-1_R R_a^T,    R_err = G R_b,
//                          x = p_b,             t = G (p_b - p_a) + P^-1_p.
// Each product is formed with the operands the constraint's kind selects,
// in the same order as for that kind alone.
template <class P>
__device__ __forceinline__ float grp_residual_pose(const ModelT<float> &m, GrpState<P> &S, const GroupPlan<P> &pl,
                                                   int c) {
  auto &E = S.u.e;
  const float(*Tf)[12] = reinterpret_cast<const float(*)[12]>(S.J);
  const bool rel = pl.crel[c] != 0;
  const int r0 = pl.croff[c], ps = pl.pslot[c], fa = pl.cfa[c], fb = pl.cfb[c];
  float Pr[9], Qr[9], Ra[9], Rb[9];
  load_R(m.cPinv[c], Pr);
  load_R(m.cQinv[c], Qr);
  const V3<float> Pp = load_p(m.cPinv[c]);
  const V3<float> Qp = load_p(m.cQinv[c]);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      Ra[r * 3 + cc] = Tf[fa][r * 4 + cc];
      Rb[r * 3 + cc] = Tf[fb][r * 4 + cc];
    }
  const V3<float> pa{Tf[fa][3], Tf[fa][7], Tf[fa][11]};
  const V3<float> pb{Tf[fb][3], Tf[fb][7], Tf[fb][11]};
  float X1[9], Y1[9], Z[9], X2[9], Y2[9], Rerr[9], G[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      X1[r * 3 + cc] = rel ? Pr[r * 3 + cc] : Ra[r * 3 + cc];
      Y1[r * 3 + cc] = rel ? Ra[cc * 3 + r] : Qr[r * 3 + cc];
    }
  mul33(X1, Y1, Z);  // pose: R_a Q^-1_R; relative pose: G
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    X2[i] = rel ? Z[i] : Pr[i];
    Y2[i] = rel ? Rb[i] : Z[i];
    G[i] = rel ? Z[i] : Pr[i];
  }
  mul33(X2, Y2, Rerr);
  const V3<float> xq = add_rot_t<7>(pa, Ra, Qp);
  const V3<float> xpt{rel ? pb.x : xq.x, rel ? pb.y : xq.y, rel ? pb.z : xq.z};
  const V3<float> tx = mulv(G, rel ? sub(pb, pa) : xq);
  const V3<float> t{tx.x + Pp.x, tx.y + Pp.y, tx.z + Pp.z};
  const auto lg = so3_log<OpsF32, float>(Rerr);
#pragma unroll
  for (int i = 0; i < 9; ++i) E.G[ps][i] = G[i];
  E.x[ps][0] = xpt.x;
  E.x[ps][1] = xpt.y;
  E.x[ps][2] = xpt.z;
  E.phi[ps][0] = lg.phi.x;
  E.phi[ps][1] = lg.phi.y;
  E.phi[ps][2] = lg.phi.z;
  E.phi[ps][3] = jl_inv_beta<float>(lg.theta, lg.s, lg.c);
  S.F[r0] = t.x;
  S.F[r0 + 1] = t.y;
  S.F[r0 + 2] = t.z;
  S.F[r0 + 3] = lg.phi.x;
  S.F[r0 + 4] = lg.phi.y;
  S.F[r0 + 5] = lg.phi.z;
  return fmaf(t.x, t.x, fmaf(t.y, t.y, fmaf(t.z, t.z, fmaf(lg.phi.x, lg.phi.x, fmaf(lg.phi.y, lg.phi.y, lg.phi.z * lg.phi.z)))));
}

// Gram phase with row blocks of RA x RB rows: every lane runs its task slots;
// each task accumulates sum_j seg(j, a) seg(j, b)^T over its joints in
// registers and stores the lower-triangular part into S.u.A.
template <int RA, int RB, class P>
__device__ __forceinline__ void grp_gram_phase(const GroupPlan<P> &pl, int ph, int g, bool go, GrpState<P> &S) {
#pragma unroll 1
  for (int t = 0; t < pl.g_nt[ph]; ++t) {
    const GrpTask tk = pl.gt[ph][g][t];
    float acc[RA][RB];
#pragma unroll
    for (int i = 0; i < RA; ++i)
#pragma unroll
      for (int k = 0; k < RB; ++k) acc[i][k] = 0.f;
    const int len = pl.g_len[ph][t];
#pragma unroll 2
    for (int s = 0; s < len; ++s) {
      if (go && s < tk.n) {
        const int j = pl.pool[tk.off + s];
        const float *sa = S.J + pl.joff[tk.a][j];
        const float *sb = S.J + pl.joff[tk.b][j];
        float va[RA], vb[RB];
#pragma unroll
        for (int i = 0; i < RA; i += 2) {
          const float2 v = lds2(sa + i);
          va[i] = v.x;
          va[i + 1] = v.y;
        }
#pragma unroll
        for (int k = 0; k < RB; k += 2) {
          const float2 v = lds2(sb + k);
          vb[k] = v.x;
          vb[k + 1] = v.y;
        }
#pragma unroll
        for (int i = 0; i < RA; ++i)
#pragma unroll
          for (int k = 0; k < RB; ++k) acc[i][k] = fmaf(va[i], vb[k], acc[i][k]);
      }
    }
    if (go && tk.n > 0) {
      const int ra = pl.croff[tk.a], rb = pl.croff[tk.b];
#pragma unroll
      for (int i = 0; i < RA; ++i)
#pragma unroll
        for (int k = 0; k < RB; ++k) {
          const int ii = ra + i, kk = rb + k;
          if (ii >= kk) S.u.A[ii * (ii + 1) / 2 + kk] = acc[i][k];
        }
    }
  }
}

// Refinement phase with row blocks of RA rows: r_a = F_a - sum_j seg(j, a) dq_j - lambda y_a.
template <int RA, class P>
__device__ __forceinline__ void grp_resid_phase(const GroupPlan<P> &pl, int ph, int g, bool go, float lambda,
                                                GrpState<P> &S) {
#pragma unroll 1
  for (int t = 0; t < pl.r_nt[ph]; ++t) {
    const GrpTask tk = pl.rt[ph][g][t];
    float acc[RA];
#pragma unroll
    for (int i = 0; i < RA; ++i) acc[i] = 0.f;
    const int len = pl.r_len[ph][t];
#pragma unroll 2
    for (int s = 0; s < len; ++s) {
      if (go && s < tk.n) {
        const int j = pl.pool[tk.off + s];
        const float *sa = S.J + pl.joff[tk.a][j];
        const float dj = S.u.s.dq[j];
#pragma unroll
        for (int i = 0; i < RA; i += 2) {
          const float2 v = lds2(sa + i);
          acc[i] = fmaf(v.x, dj, acc[i]);
          acc[i + 1] = fmaf(v.y, dj, acc[i + 1]);
        }
      }
    }
    if (go && tk.n > 0) {
      const int ra = pl.croff[tk.a];
#pragma unroll
      for (int i = 0; i < RA; ++i) S.F[ra + i] = fmaf(-lambda, S.u.s.y[ra + i], S.F[ra + i] - acc[i]);
    }
  }
}

// One FP32 iteration for the group's configuration.  All lanes of the warp
// call it together (it holds warp-wide synchronisation); `act` says whether
// this group has a configuration.  Returns true for a group whose
// configuration leaves the FP32 loop (flags say why).
template <class P, class A>
__device__ __forceinline__ bool grp_iter(const A &a, const GrpTables<P> &tb, const GroupPlan<P> &pl,
                                         GrpState<P> &S, bool act, int &it, uint32_t &fl) {
  constexpr int K = kdim<P>(), NC = P::NC;
  constexpr int MR = (K + GG - 1) / GG;  // rows per lane
  const int lane = threadIdx.x & 31;
  const int g = lane & (GG - 1);
  const int base = lane & ~(GG - 1);
  const ModelT<float> &m = a.m;
  auto &E = S.u.e;

  // 1. FK along the lane's schedule
  {
    float T[12], S0[12], S1[12];
#pragma unroll
    for (int e = 0; e < 12; ++e) T[e] = S0[e] = S1[e] = 0.f;
    // the prismatic root chain in closed form: constant rotations, origins
    // pre_c[i] + sum_{k <= i} q_k pre_a[k]
    const int n_pre = pl.n_pre;
    if (n_pre > 0 && act) {
      float o0 = 0.f, o1 = 0.f, o2 = 0.f;
#pragma unroll
      for (int i = 0; i < GMAX_PRE; ++i) {
        if (i < n_pre) {
          const float qi = S.q[i];
          o0 = fmaf(qi, tb.pre_a[i][0], o0);
          o1 = fmaf(qi, tb.pre_a[i][1], o1);
          o2 = fmaf(qi, tb.pre_a[i][2], o2);
          const float x0 = tb.pre_c[i][0] + o0, x1 = tb.pre_c[i][1] + o1, x2 = tb.pre_c[i][2] + o2;
          if (pl.fk_store[g][i]) {
            E.zo[i][0] = tb.pre_a[i][0];
            E.zo[i][1] = tb.pre_a[i][1];
            E.zo[i][2] = tb.pre_a[i][2];
            E.zo[i][3] = x0;
            E.zo[i][4] = x1;
            E.zo[i][5] = x2;
            const float mi = tb.mass[i];
            S.C(i)[0] = fmaf(mi, x0, tb.pre_mc[i][0]);
            S.C(i)[1] = fmaf(mi, x1, tb.pre_mc[i][1]);
            S.C(i)[2] = fmaf(mi, x2, tb.pre_mc[i][2]);
          }
          if (i == n_pre - 1) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
#pragma unroll
              for (int cc = 0; cc < 3; ++cc) T[r * 4 + cc] = tb.pre_R[i][r * 3 + cc];
            }
            T[3] = x0;
            T[7] = x1;
            T[11] = x2;
          }
        }
      }
    }
#pragma unroll 1
    for (int k = n_pre; k < pl.n_fk; ++k) {
      const int j = pl.fk_j[g][k];
      if (act && j >= 0) {
        const int par = pl.fk_par[g][k];
        if (par != 0) {  // a root or a branch point: the parent frame is not the last one
#pragma unroll
          for (int e = 0; e < 12; ++e) {
            const float id = (e == 0 || e == 5 || e == 10) ? 1.f : 0.f;
            T[e] = par == 1 ? S0[e] : (par == 2 ? S1[e] : id);
          }
        }
        const float *X = tb.X[j];
        float Lc[12];
        const float qj = S.q[j];
        if (tb.rev[j]) {
          float sn, cs;
          sincos_f32(qj, sn, cs);
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            Lc[r * 4] = fmaf(cs, X[r * 4], sn * X[r * 4 + 1]);
            Lc[r * 4 + 1] = fmaf(cs, X[r * 4 + 1], -(sn * X[r * 4]));
            Lc[r * 4 + 2] = X[r * 4 + 2];
            Lc[r * 4 + 3] = X[r * 4 + 3];
          }
        } else {
#pragma unroll
          for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int c = 0; c < 3; ++c) Lc[r * 4 + c] = X[r * 4 + c];
            Lc[r * 4 + 3] = fmaf(qj, X[r * 4 + 2], X[r * 4 + 3]);
          }
        }
        {
          float Tn[12];
          compose34(T, Lc, Tn);
#pragma unroll
          for (int e = 0; e < 12; ++e) T[e] = Tn[e];
        }
        const int sv = pl.fk_save[g][k];
        if (sv >= 0) {
#pragma unroll
          for (int e = 0; e < 12; ++e) {
            if (sv == 0) S0[e] = T[e];
            else S1[e] = T[e];
          }
        }
        if (pl.fk_store[g][k]) {
          E.zo[j][0] = T[2];
          E.zo[j][1] = T[6];
          E.zo[j][2] = T[10];
          E.zo[j][3] = T[3];
          E.zo[j][4] = T[7];
          E.zo[j][5] = T[11];
          const float *cm = tb.com[j];  // local link CoM
          const float mj = tb.mass[j];
#pragma unroll
          for (int r = 0; r < 3; ++r)
            S.C(j)[r] = mj * fmaf(T[r * 4], cm[0], fmaf(T[r * 4 + 1], cm[1], fmaf(T[r * 4 + 2], cm[2], T[r * 4 + 3])));
          int f = -1;  // the task frame on this link, if any (one copy of the composition)
          static_for<P::NF>([&](auto FF) {
            if (j == P::frame_link(decltype(FF)::value)) f = decltype(FF)::value;
          });
          if (f >= 0) {
            float Fx[12], To[12];
#pragma unroll
            for (int e = 0; e < 12; ++e) Fx[e] = tb.fX[f][e];
            compose34(T, Fx, To);
#pragma unroll
            for (int e = 0; e < 12; ++e) S.J[f * 12 + e] = To[e];
          }
        }
      }
    }
  }
  __syncwarp();
  // 2. subtree moments: limbs on their lanes, then the trunk on lane 0
  float tot[3] = {0.f, 0.f, 0.f};
  if constexpr (needs_com<P>()) {
#pragma unroll 1
    for (int k = 0; k < pl.n_cb; ++k) {
      const int j = pl.cb_j[g][k];
      if (act && j >= 0) {
        float c0 = S.C(j)[0], c1 = S.C(j)[1], c2 = S.C(j)[2];
#pragma unroll
        for (int h = 0; h < GMAX_CH; ++h) {
          const int cj = pl.child[j][h];
          if (cj >= 0) {
            c0 += S.C(cj)[0];
            c1 += S.C(cj)[1];
            c2 += S.C(cj)[2];
          }
        }
        S.C(j)[0] = c0;
        S.C(j)[1] = c1;
        S.C(j)[2] = c2;
      }
    }
    __syncwarp();
    if (act && g == 0) {
#pragma unroll 1
      for (int k = 0; k < pl.n_cr; ++k) {
        const int j = pl.cr_j[k];
        float c0 = S.C(j)[0], c1 = S.C(j)[1], c2 = S.C(j)[2];
#pragma unroll
        for (int h = 0; h < GMAX_CH; ++h) {
          const int cj = pl.child[j][h];
          if (cj >= 0) {
            c0 += S.C(cj)[0];
            c1 += S.C(cj)[1];
            c2 += S.C(cj)[2];
          }
        }
        S.C(j)[0] = c0;
        S.C(j)[1] = c1;
        S.C(j)[2] = c2;
      }
    }
    __syncwarp();
#pragma unroll 1
    for (int k = 0; k < pl.n_roots; ++k) {
      const int rj = pl.roots[k];
      tot[0] += S.C(rj)[0];
      tot[1] += S.C(rj)[1];
      tot[2] += S.C(rj)[2];
    }
  }
  // 3. residuals: constraint c on lane c mod 4; the pose-like ones share one
  // code path (run time), the others have their own (compile time)
  float r2p = 0.f;
  if constexpr (grp_npose<P>() > 0) {
#pragma unroll 1
    for (int c = g; c < NC; c += GG)
      if (act && pl.pslot[c] >= 0) r2p += grp_residual_pose<P>(m, S, pl, c);
  }
  static_for<NC>([&](auto CC) {
    constexpr int c = decltype(CC)::value;
    if constexpr (!grp_pose_like<P>(c)) {
      if (act && g == (c % GG)) r2p += grp_residual<P, c>(m, S, tot);
    }
  });
  const float r2 = grp_sum(r2p);
  bool done = false;
  if (act) {
    if (!(r2 <= FLT_MAX)) {
      fl |= FL_NONFINITE;
      done = true;
    } else if (r2 < a.tol2 && !(fl & FL_INT_FORCE)) {
      fl |= FL_INT_FP32CONV;
      done = true;
    } else if (it >= a.cap) {
      fl |= FL_CAP;
      done = true;
    }
  }
  const bool go = act && !done;
  __syncwarp();
  // 4. Jacobian segments: the 2-row ones first (they read the subtree
  // moments, which the 6-row segments overwrite)
#pragma unroll 1
  for (int k = 0; k < pl.n_j2; ++k) {
    const int j = pl.j2_j[g][k];
    if (go && j >= 0) {
      const int c = pl.j2_c[g][k];
      const float sg = static_cast<float>(tb.sgn[c][j]);
      const V3<float> z{E.zo[j][0], E.zo[j][1], E.zo[j][2]};
      const V3<float> o{E.zo[j][3], E.zo[j][4], E.zo[j][5]};
      const bool rev = tb.rev[j] != 0;
      const float Mj = tb.msub[j];
      const float *Cj = S.C(j);
      const V3<float> rr{fmaf(-Mj, o.x, Cj[0]), fmaf(-Mj, o.y, Cj[1]), fmaf(-Mj, o.z, Cj[2])};
      const V3<float> d = cross(z, rr);
      const float fpr = Mj * m.inv_mass;
      float g0 = sg * (rev ? d.x * m.inv_mass : fpr * z.x);
      float g1 = sg * (rev ? d.y * m.inv_mass : fpr * z.y);
      if (pl.chull[c]) {  // inside: 0; on an edge: n n^T g; at a vertex: g
        const int hs = pl.hslot[c];
        const int hm = E.hmode[hs];
        if (hm == 0) {
          g0 = g1 = 0.f;
        } else if (hm == 1) {
          const float sd = fmaf(E.hn[hs][0], g0, E.hn[hs][1] * g1);
          g0 = E.hn[hs][0] * sd;
          g1 = E.hn[hs][1] * sd;
        }
      }
      float *dst = S.J + pl.joff[c][j];
      dst[0] = g0;
      dst[1] = g1;
    }
  }
  __syncwarp();
#pragma unroll 1
  for (int k = 0; k < pl.n_j6; ++k) {
    const int j = pl.j6_j[g][k];
    if (go && j >= 0) {
      const int c = pl.j6_c[g][k];
      const float sg = static_cast<float>(tb.sgn[c][j]);
      const V3<float> z{E.zo[j][0], E.zo[j][1], E.zo[j][2]};
      const V3<float> o{E.zo[j][3], E.zo[j][4], E.zo[j][5]};
      float G[9];
      const int ps = pl.pslot[c];
#pragma unroll
      for (int i = 0; i < 9; ++i) G[i] = E.G[ps][i];
      const bool rev = tb.rev[j] != 0;
      const V3<float> xp{E.x[ps][0], E.x[ps][1], E.x[ps][2]};
      const V3<float> v = rev ? cross(z, sub(xp, o)) : z;
      const V3<float> vt = mulv(G, v);
      const V3<float> w = jl_inv_apply(V3<float>{E.phi[ps][0], E.phi[ps][1], E.phi[ps][2]}, E.phi[ps][3], mulv(G, z));
      float *dst = S.J + pl.joff[c][j];
      dst[0] = sg * vt.x;
      dst[1] = sg * vt.y;
      dst[2] = sg * vt.z;
      dst[3] = rev ? sg * w.x : 0.f;
      dst[4] = rev ? sg * w.y : 0.f;
      dst[5] = rev ? sg * w.z : 0.f;
    }
  }
  __syncwarp();
  // 5. Gram blocks (overwrites the FK / residual data)
  grp_gram_phase<6, 6>(pl, 0, g, go, S);
  grp_gram_phase<6, 2>(pl, 1, g, go, S);
  grp_gram_phase<2, 6>(pl, 2, g, go, S);
  grp_gram_phase<2, 2>(pl, 3, g, go, S);
  // diagonal blocks of 2-row constraints: every joint, over the dq partition
  static_for<NC>([&](auto CC) {
    constexpr int c = decltype(CC)::value;
    if constexpr (grp_com_like<P>(c)) {
      constexpr int r0 = roff<P>(c);
      float s00 = 0.f, s10 = 0.f, s11 = 0.f;
#pragma unroll 1
      for (int k = 0; k < pl.n_dq; ++k) {
        const int j = pl.dq_j[g][k];
        const int o = j >= 0 ? pl.joff[c][j] : -1;
        if (go && o >= 0) {
          const float2 v = lds2(S.J + o);
          s00 = fmaf(v.x, v.x, s00);
          s10 = fmaf(v.y, v.x, s10);
          s11 = fmaf(v.y, v.y, s11);
        }
      }
      s00 = grp_sum(s00);
      s10 = grp_sum(s10);
      s11 = grp_sum(s11);
      if (go && g == 0) {
        S.u.A[r0 * (r0 + 1) / 2 + r0] = s00;
        S.u.A[(r0 + 1) * (r0 + 2) / 2 + r0] = s10;
        S.u.A[(r0 + 1) * (r0 + 2) / 2 + r0 + 1] = s11;
      }
    }
  });
  __syncwarp();
  // 6. Cholesky: rows i = 4 mm + g in registers (row i has entries 0..i)
  float L[MR][GG * MR];
  float invd[MR];
#pragma unroll
  for (int mm = 0; mm < MR; ++mm) {
    const int i = GG * mm + g;
    const uint32_t am = pl.amask[i < K ? i : 0];
    invd[mm] = 0.f;
#pragma unroll
    for (int b = 0; b < GG * (mm + 1); ++b) {
      float v = 0.f;
      if (go && i < K && b <= i && ((am >> b) & 1u)) v = S.u.A[i * (i + 1) / 2 + b];
      if (b == i) v += a.lambda;
      L[mm][b] = v;
    }
  }
  __syncwarp();
  float minpiv = FLT_MAX;
  static_for<K>([&](auto KK) {
    constexpr int k = decltype(KK)::value;
    const int ow = k % GG, mk = k / GG;
    const float piv = __shfl_sync(FULL, L[mk][k], base + ow);
    minpiv = fminf(minpiv, piv);
    const float ik = rsqrtf(piv);
    float *col = S.u.s.Lc + lcol_base<K>(k);
#pragma unroll
    for (int mm = mk; mm < MR; ++mm) {
      const int i = GG * mm + g;
      if (i == k) {
        invd[mm] = ik;
        L[mm][k] = piv * ik;
      } else if (i > k && i < K) {
        L[mm][k] *= ik;
      }
      if (go && i >= k && i < K) col[i - k] = L[mm][k];
    }
    __syncwarp();
    if (k + 1 < K) {
      // column k below the diagonal, rows k+1 .. K-1
      float cv[K];
#pragma unroll
      for (int b = k + 1; b < K; ++b) cv[b] = go ? col[b - k] : 0.f;
      static_for<MR>([&](auto MMc) {
        constexpr int mm = decltype(MMc)::value;
        if constexpr (mm >= (k + 1) / GG && !l_col_block_zero<P, mm, k>()) {
          const int i = GG * mm + g;
          const float lik = L[mm][k];
#pragma unroll
          for (int b = k + 1; b < GG * (mm + 1) && b < K; ++b)
            if (i > k && b <= i) L[mm][b] = fmaf(-lik, cv[b], L[mm][b]);
        }
      });
    }
  });
  if (go && !(minpiv >= a.pivot)) {  // includes NaN: this configuration continues in FP64
    fl |= FL_INT_NEEDS_F64;
    done = true;
  }
  const bool go2 = act && !done;
  int colo[MR];  // start of column 4 mm + g of L
#pragma unroll
  for (int mm = 0; mm < MR; ++mm) colo[mm] = pl.lcol[(GG * mm + g) < K ? GG * mm + g : 0];
  // (L L^T)^{-1} b for rows held by the lanes (t[mm] = b_{4 mm + g})
  auto subst = [&](float (&t)[MR]) {
    static_for<K>([&](auto KK) {  // forward: L y = b
      constexpr int k = decltype(KK)::value;
      constexpr int ow = k % GG, mk = k / GG;
      const float yk = __shfl_sync(FULL, t[mk] * invd[mk], base + ow);
      static_for<MR>([&](auto MMc) {
        constexpr int mm = decltype(MMc)::value;
        if constexpr (mm >= mk && !l_col_block_zero<P, mm, k>()) {
          const int i = GG * mm + g;
          if (i == k) t[mm] = yk;
          else if (i > k) t[mm] = fmaf(-L[mm][k], yk, t[mm]);
        }
      });
    });
    static_for<K>([&](auto KB) {  // back: L^T x = y, L[k][i] from column i
      constexpr int k = K - 1 - decltype(KB)::value;
      constexpr int ow = k % GG, mk = k / GG;
      const float xk = __shfl_sync(FULL, t[mk] * invd[mk], base + ow);
      static_for<MR>([&](auto MMc) {
        constexpr int mm = decltype(MMc)::value;
        if constexpr (mm <= mk && !l_row_seg_zero<P, k, mm>()) {
          const int i = GG * mm + g;
          if (i == k) {
            t[mm] = xk;
          } else if (i < k) {
            // L[k][i]: row k of column i
            const float l = go2 ? S.u.s.Lc[colo[mm] + (k - i)] : 0.f;
            t[mm] = fmaf(-l, xk, t[mm]);
          }
        }
      });
    });
  };
  // dq = J^T y for the lane's dq joints (y from shared memory)
  auto jt_y = [&]() {
    float yv[K];
#pragma unroll
    for (int i = 0; i < K; ++i) yv[i] = go2 ? S.u.s.y[i] : 0.f;
#pragma unroll 1
    for (int k = 0; k < pl.n_dq; ++k) {
      const int j = pl.dq_j[g][k];
      if (go2 && j >= 0) {
        float acc = 0.f;
        static_for<NC>([&](auto CC) {
          constexpr int c = decltype(CC)::value;
          constexpr int rc = cdim(P::ckind(c));
          constexpr int r0 = roff<P>(c);
          const int o = pl.joff[c][j];
          if (o >= 0) {
#pragma unroll
            for (int i = 0; i < rc; i += 2) {
              const float2 v = lds2(S.J + o + i);
              acc = fmaf(v.x, yv[r0 + i], fmaf(v.y, yv[r0 + i + 1], acc));
            }
          }
        });
        S.u.s.dq[j] = acc;
      }
    }
  };
  // y = A^{-1} F, then one refinement step with the residual from J,
  // r = F - J (J^T y) - lambda y: y += A^{-1} r.  Both passes run the same
  // code (a loop, not two inlined copies).
  float t[MR], ty[MR];
#pragma unroll
  for (int mm = 0; mm < MR; ++mm) {
    const int i = GG * mm + g;
    t[mm] = (go2 && i < K) ? S.F[i] : 0.f;
    ty[mm] = 0.f;
  }
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    subst(t);
#pragma unroll
    for (int mm = 0; mm < MR; ++mm) {
      const int i = GG * mm + g;
      ty[mm] += t[mm];
      if (go2 && i < K) S.u.s.y[i] = ty[mm];
    }
    __syncwarp();
    jt_y();
    __syncwarp();
    if (pass == 1) break;
    grp_resid_phase<6>(pl, 0, g, go2, a.lambda, S);
    static_for<NC>([&](auto CC) {  // 2-row blocks: every joint, over the dq partition
      constexpr int c = decltype(CC)::value;
      if constexpr (grp_com_like<P>(c)) {
        constexpr int r0 = roff<P>(c);
        float s0 = 0.f, s1 = 0.f;
#pragma unroll 1
        for (int k = 0; k < pl.n_dq; ++k) {
          const int j = pl.dq_j[g][k];
          const int o = j >= 0 ? pl.joff[c][j] : -1;
          if (go2 && o >= 0) {
            const float2 v = lds2(S.J + o);
            const float dj = S.u.s.dq[j];
            s0 = fmaf(v.x, dj, s0);
            s1 = fmaf(v.y, dj, s1);
          }
        }
        s0 = grp_sum(s0);
        s1 = grp_sum(s1);
        if (go2 && g == 0) {
          S.F[r0] = fmaf(-a.lambda, S.u.s.y[r0], S.F[r0] - s0);
          S.F[r0 + 1] = fmaf(-a.lambda, S.u.s.y[r0 + 1], S.F[r0 + 1] - s1);
        }
      }
    });
    __syncwarp();
#pragma unroll
    for (int mm = 0; mm < MR; ++mm) {
      const int i = GG * mm + g;
      t[mm] = (go2 && i < K) ? S.F[i] : 0.f;
    }
    __syncwarp();
  }
  // alpha, MaxDistance, update
  float s2p = 0.f;
#pragma unroll 1
  for (int k = 0; k < pl.n_dq; ++k) {
    const int j = pl.dq_j[g][k];
    if (go2 && j >= 0) {
      const float d = S.u.s.dq[j] * a.alpha;
      S.u.s.dq[j] = d;
      s2p = fmaf(d, d, s2p);
    }
  }
  const float s2 = grp_sum(s2p);
  if (go2 && a.max_step2 > 0.f && s2 > a.max_step2) {
    fl |= FL_DIV;
    done = true;
  }
  const bool go3 = act && !done;
#pragma unroll 1
  for (int k = 0; k < pl.n_dq; ++k) {
    const int j = pl.dq_j[g][k];
    if (go3 && j >= 0) S.q[j] -= S.u.s.dq[j];
  }
  if (go3) {
    ++it;
    fl &= ~FL_INT_FORCE;
    if (!(s2 <= FLT_MAX)) {
      fl |= FL_NONFINITE;
      done = true;
    }
  }
  __syncwarp();
  return act && done;
}

template <class P, int W>
__global__ void __launch_bounds__(W * 32, 1) k_project_group(const __grid_constant__ GroupArgs<P> a) {
  constexpr int D = P::D;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GrpShared<P> &sh = *reinterpret_cast<GrpShared<P> *>(smem_raw);
  unsigned char *ws = smem_raw + ((sizeof(GrpShared<P>) + 15) & ~size_t(15));
  __shared__ int s_item[W][40];  // parked configurations: < 32 + 8 (the launcher keeps totals below 2^31)
  __shared__ uint32_t s_meta[W][40];
  __shared__ int s_ritem[W][RETRY_CAP];  // sent back to the FP32 loop by the acceptance
  __shared__ uint32_t s_rmeta[W][RETRY_CAP];
  {
    static_assert(sizeof(GrpTables<P>) % 4 == 0 && sizeof(GroupPlan<P>) % 4 == 0, "word copies");
    const int *src = reinterpret_cast<const int *>(&a.t);
    int *dst = reinterpret_cast<int *>(&sh.tb);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(GrpTables<P>) / 4); i += blockDim.x) dst[i] = src[i];
    const int *src2 = reinterpret_cast<const int *>(&a.pl);
    int *dst2 = reinterpret_cast<int *>(&sh.pl);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(GroupPlan<P>) / 4); i += blockDim.x) dst2[i] = src2[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int g = lane & (GG - 1);
  const int grp = lane >> 2;
  GrpState<P> &S = *reinterpret_cast<GrpState<P> *>(ws + (wib * GCPW + grp) * grp_state_stride<P>());
  long long qn = 0, qe = 0;  // warp-local queue [qn, qe)
  bool more = true;
  bool act = false;
  long long item = 0;
  int it = 0;
  uint32_t fl = 0;
  int pend = 0;
  int nret = 0;  // warp-uniform count of configurations to retry in FP32
  const unsigned lead = 0x11111111u;  // lane 0 of every group
  while (true) {
    // refill idle groups (decided by each group's lane 0, shared by the
    // group): retries first, then new work
    const unsigned idle = __ballot_sync(FULL, !act) & lead;
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
        if (static_cast<long long>(b) >= a.total) {
          more = false;
        } else {
          b0 = static_cast<long long>(b);
          b1 = b0 + a.chunk < a.total ? b0 + a.chunk : a.total;
        }
      }
      const int rank_all = __popc(idle & ((1u << (grp * GG)) - 1u));
      if (!act) {
        if (rank_all < from_r) {  // one more FP32 step from the parked iterate
          const int pos = nret - 1 - rank_all;
          item = s_ritem[wib][pos];
          const uint32_t meta = s_rmeta[wib][pos];
          it = static_cast<int>(meta & 0xffu);
          fl = ((meta >> 8) & ~(FL_INT_FP32CONV | FL_INT_NEEDS_F64)) | FL_INT_FORCE;
          act = true;
          for (int j = g; j < D; j += GG) S.q[j] = MCP_CHK(item, a.ld_out) ? a.q_out[j * a.ld_out + item] : 0.f;
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
            for (int j = g; j < D; j += GG) S.q[j] = MCP_CHK(item, a.src.ld) ? a.src.q[j * a.src.ld + item] : 0.f;
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
    __syncwarp();
    const bool done = grp_iter<P>(a, sh.tb, sh.pl, S, act, it, fl);
    // park finished configurations
    const unsigned fin = __ballot_sync(FULL, done) & lead;
    if (fin != 0u) {
      if (done) {
        if (MCP_CHK(item, a.ld_out))
          for (int j = g; j < D; j += GG) a.q_out[j * a.ld_out + item] = S.q[j];
        if (g == 0) {
          const int pos = pend + __popc(fin & ((1u << lane) - 1u));
          s_item[wib][pos] = static_cast<int>(item);
          s_meta[wib][pos] = static_cast<uint32_t>(it) | (fl << 8);
        }
        act = false;
      }
      pend += __popc(fin);
      __syncwarp();
    }
    const bool drained = !__any_sync(FULL, act) && qn >= qe && !more && nret == 0;
    // FP64 acceptance, one configuration per lane, 32 at a time; a failed
    // acceptance with steps left goes back to the FP32 loop
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
        retry = accept_one<P, FORM_STACKED>(a, it_item, static_cast<int>(meta & 0xffu), meta >> 8, room);
      }
      const unsigned rm = __ballot_sync(FULL, retry);
      __syncwarp();
      if (retry) {
        const int rp = nret + __popc(rm & ((1u << lane) - 1u));
        s_ritem[wib][rp] = static_cast<int>(it_item);
        s_rmeta[wib][rp] = meta;
      }
      nret += __popc(rm);
      pend -= take;
      __syncwarp();
    }
    if (drained && pend == 0 && nret == 0) break;
  }
}

template <class P>
size_t group_smem_bytes(int W) {
  return ((sizeof(GrpShared<P>) + 15) & ~size_t(15)) + static_cast<size_t>(W) * GCPW * grp_state_stride<P>();
}

template <class P>
cudaError_t launch_project_group(const HostModel &hm, const ProjCall &c, int *launches) {
  static_assert(grp_supported<P>(), "the group kernel takes trees with pose-like and CoM-like constraints");
  if (c.total <= 0) return cudaSuccess;
  if (c.precision == 1 || c.segments || c.outer || c.cyclic) return cudaErrorNotSupported;
  if (c.total > 0x7fffffffLL) return cudaErrorInvalidValue;  // parked indices are 32-bit
  constexpr int W = 11;  // one block per SM: 88 configurations, bounded by shared memory
  struct Planned {
    GroupPlan<P> plan;
    bool ok;
  };
  static const Planned pp = [] {  // once per class (thread-safe initialisation)
    Planned h{};
    h.ok = make_group_plan<P>(h.plan, nullptr);
    return h;
  }();
  if (!pp.ok) return cudaErrorNotSupported;
  GroupArgs<P> a;
  cudaError_t err = cudaMemsetAsync(c.counter, 0, sizeof(unsigned long long), c.stream);
  if (err != cudaSuccess) return err;
  a.m = hm.m32;
  a.t = make_grp_tables<P>(hm.m32, hm.m64);
  a.pl = pp.plan;
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
  a.chunk = 16;
  a.cap = c.cap;
  a.tol2 = static_cast<float>(c.tol * c.tol);
  a.lambda = static_cast<float>(c.lambda);
  a.max_step2 = c.max_step > 0 ? static_cast<float>(c.max_step * c.max_step) : 0.f;
  a.pivot = static_cast<float>(c.pivot);
  a.tol2_64 = c.tol * c.tol;
  a.lambda64 = c.lambda;
  a.alpha = static_cast<float>(c.alpha);
  auto kern = k_project_group<P, W>;
  const size_t smem = group_smem_bytes<P>(W);
  err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorNotSupported;
  long long blocks = static_cast<long long>(hm.sm_count) * per_sm;
  const long long need = (c.total + static_cast<long long>(GCPW) * W - 1) / (static_cast<long long>(GCPW) * W);
  if (blocks > need) blocks = need;
  kern<<<static_cast<unsigned>(blocks), W * 32, smem, c.stream>>>(a);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace mcp
