// Host-side consistency check of the work plan of the group-cooperative
// humanoid kernel (four lanes per configuration): every joint is placed by
// forward kinematics exactly once with its parent available, every subtree
// CoM sum comes after its children, every structurally nonzero Jacobian
// segment (joint, constraint) and every nonzero Gram block is assigned to
// exactly one lane with the right joint set, the refinement tasks and the dq
// partition cover every joint once, the Gram mask matches what the tasks
// write, the compile-time zero pattern of the Cholesky factor (the blocks
// the kernel skips) matches a double-precision factor, and the prismatic root
// prefix placed in closed form matches a step-by-step composition.  Runs on the CPU (no kernel is launched); prints "<class>: N
// problems" per class and exits with the total.
#include <cmath>
#include <cstdio>
#include <set>
#include "../../paper_2604_13323_gb300/csrc/mcp_group.cuh"
#include "../../paper_2604_13323_gb300/csrc/mcp_problems.cuh"
using namespace mcp;
template <class P> int check() {
  GroupPlan<P> pl; const char *why = nullptr;
  if (!make_group_plan<P>(pl, &why)) { printf("plan failed: %s\n", why); return 1; }
  constexpr int D = P::D, NC = P::NC, K = kdim<P>();
  int bad = 0;
  printf("%s: n_fk=%d n_cb=%d n_cr=%d roots=%d n_j6=%d n_j2=%d n_dq=%d\n", P::name, pl.n_fk, pl.n_cb, pl.n_cr, pl.n_roots, pl.n_j6, pl.n_j2, pl.n_dq);
  // FK: every joint stored exactly once; parents available
  int stored[D] = {0};
  for (int g = 0; g < GG; ++g) {
    std::set<int> have; int prev = -1; int slot[2] = {-1, -1};
    printf(" lane %d FK:", g);
    for (int k = 0; k < GMAX_FK; ++k) {
      int j = pl.fk_j[g][k]; if (j < 0) continue;
      printf(" %d(p%d s%d w%d)", j, pl.fk_par[g][k], pl.fk_save[g][k], pl.fk_store[g][k]);
      int p = P::parent(j), par = pl.fk_par[g][k];
      if (par == 3 && p != -1) bad++, printf("[bad root]");
      if (par == 0 && prev != p) bad++, printf("[bad prev]");
      if ((par == 1 || par == 2) && slot[par - 1] != p) bad++, printf("[bad slot]");
      if (pl.fk_save[g][k] >= 0) slot[pl.fk_save[g][k]] = j;
      if (pl.fk_store[g][k]) stored[j]++;
      prev = j; have.insert(j);
      if (k >= pl.n_fk) bad++;
    }
    printf("\n");
  }
  for (int j = 0; j < D; ++j) if (stored[j] != 1) bad++, printf("joint %d stored %d\n", j, stored[j]);
  // the prismatic root prefix placed in closed form: a chain of prismatic
  // joints from the root, at the head of every lane's schedule, nothing saved
  // in it and no task frame on it; the step after it continues from it
  printf(" prismatic prefix: %d joints\n", pl.n_pre);
  if (pl.n_pre < 0 || pl.n_pre > GMAX_PRE) bad++;
  for (int k = 0; k < pl.n_pre; ++k) {
    if (P::jtype(k) != PRIS || P::parent(k) != k - 1) bad++, printf("prefix joint %d\n", k);
    for (int g = 0; g < GG; ++g) if (pl.fk_j[g][k] != k || pl.fk_save[g][k] >= 0) bad++, printf("prefix step %d lane %d\n", k, g);
  }
  for (int f = 0; f < P::NF; ++f) if (P::frame_link(f) < pl.n_pre) bad++;
  for (int g = 0; g < GG; ++g) if (pl.n_pre > 0 && pl.fk_j[g][pl.n_pre] >= 0 && pl.fk_par[g][pl.n_pre] != 0) bad++;
  // its constants against a step-by-step composition of a random model
  if (pl.n_pre > 0) {
    static ModelT<double> m64{};
    static ModelT<float> m32{};
    unsigned long long x = 0x2545F4914F6CDD1Dull;
    auto rnd = [&]() { x ^= x << 13; x ^= x >> 7; x ^= x << 17; return (double)(x >> 11) / 9007199254740992.0 - 0.5; };
    for (int j = 0; j < D; ++j) {
      const double a = 3.0 * rnd(), c = std::cos(a), s_ = std::sin(a);   // a rotation about x, then a translation
      const double Xr[12] = {1, 0, 0, rnd(), 0, c, -s_, rnd(), 0, s_, c, rnd()};
      for (int e = 0; e < 12; ++e) m64.X[j][e] = Xr[e];
      m64.mass[j] = 1.0 + rnd();
      for (int r = 0; r < 3; ++r) m64.com[j][r] = 0.1 * rnd();
    }
    const GrpTables<P> tb = make_grp_tables<P>(m32, m64);
    double q[GMAX_PRE];
    for (int i = 0; i < GMAX_PRE; ++i) q[i] = rnd();
    double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, pp[3] = {0, 0, 0}, acc[3] = {0, 0, 0};
    for (int i = 0; i < pl.n_pre; ++i) {
      double Rn[9], pn[3];   // T_i = T_{i-1} X_i Tz(q_i)
      for (int r = 0; r < 3; ++r) {
        for (int cc = 0; cc < 3; ++cc) Rn[r * 3 + cc] = R[r * 3] * m64.X[i][cc] + R[r * 3 + 1] * m64.X[i][4 + cc] + R[r * 3 + 2] * m64.X[i][8 + cc];
        pn[r] = pp[r] + R[r * 3] * m64.X[i][3] + R[r * 3 + 1] * m64.X[i][7] + R[r * 3 + 2] * m64.X[i][11];
      }
      for (int r = 0; r < 3; ++r) pn[r] += q[i] * Rn[r * 3 + 2];
      for (int e = 0; e < 9; ++e) R[e] = Rn[e];
      for (int r = 0; r < 3; ++r) pp[r] = pn[r];
      double err = 0;
      for (int r = 0; r < 3; ++r) {
        acc[r] += q[i] * tb.pre_a[i][r];
        err = std::max(err, std::fabs(tb.pre_c[i][r] + acc[r] - pp[r]));
        err = std::max(err, std::fabs(tb.pre_a[i][r] - R[r * 3 + 2]));
        const double mc = m64.mass[i] * (R[r * 3] * m64.com[i][0] + R[r * 3 + 1] * m64.com[i][1] + R[r * 3 + 2] * m64.com[i][2]);
        err = std::max(err, std::fabs(tb.pre_mc[i][r] - mc));
      }
      for (int e = 0; e < 9; ++e) err = std::max(err, std::fabs(tb.pre_R[i][e] - R[e]));
      if (err > 1e-6) bad++, printf("prefix joint %d constants off by %g\n", i, err);
    }
  }
  // CoM: every joint exactly once in own/trunk lists; children processed before
  int seen[D] = {0};
  for (int g = 0; g < GG; ++g) { std::set<int> done; for (int k = 0; k < GMAX_CB; ++k) { int j = pl.cb_j[g][k]; if (j < 0) continue; seen[j]++; for (int h = 0; h < GMAX_CH; ++h) { int c = pl.child[j][h]; if (c >= 0 && !done.count(c)) bad++, printf("own child %d of %d not done on lane %d\n", c, j, g); } done.insert(j); if (k >= pl.n_cb) bad++; } }
  { std::set<int> done; for (int k = 0; k < GMAX_CR; ++k) { int j = pl.cr_j[k]; if (j < 0) continue; seen[j]++; done.insert(j); if (k >= pl.n_cr) bad++; } }
  for (int j = 0; j < D; ++j) if (seen[j] != 1) bad++, printf("joint %d in CoM lists %d times\n", j, seen[j]);
  // segments: each (j,c) with col_sign != 0 exactly once; offsets in range, even
  int segseen[NC][D] = {{0}};
  for (int g = 0; g < GG; ++g) for (int k = 0; k < GMAX_JI; ++k) {
    if (pl.j6_j[g][k] >= 0) { int j = pl.j6_j[g][k], c = pl.j6_c[g][k]; segseen[c][j]++; if (!grp_pose_like<P>(c)) bad++; if (k >= pl.n_j6) bad++; }
    if (pl.j2_j[g][k] >= 0) { int j = pl.j2_j[g][k], c = pl.j2_c[g][k]; segseen[c][j]++; if (!grp_com_like<P>(c)) bad++; if (k >= pl.n_j2) bad++; }
  }
  constexpr int NJ = GrpState<P>::NJ;
  for (int c = 0; c < NC; ++c) for (int j = 0; j < D; ++j) {
    bool nz = col_sign<P>(c, j) != 0;
    if (segseen[c][j] != (nz ? 1 : 0)) bad++, printf("seg (%d,%d) seen %d\n", j, c, segseen[c][j]);
    if (nz && (pl.joff[c][j] < 0 || pl.joff[c][j] % 2 || pl.joff[c][j] + cdim(P::ckind(c)) > grp_nseg_floats<P>())) bad++, printf("joff bad\n");
    if (!nz && pl.joff[c][j] != -1) bad++;
  }
  // dq joints exactly once
  int dqs[D] = {0};
  for (int g = 0; g < GG; ++g) for (int k = 0; k < GMAX_DQ; ++k) if (pl.dq_j[g][k] >= 0) { dqs[pl.dq_j[g][k]]++; if (k >= pl.n_dq) bad++; }
  for (int j = 0; j < D; ++j) if (dqs[j] != 1) bad++, printf("dq joint %d: %d\n", j, dqs[j]);
  // Gram: every nonzero lower block exactly once, joint lists = intersections
  int blk[NC][NC] = {{0}};
  for (int ph = 0; ph < 4; ++ph) {
    printf(" phase %d: nt=%d len=", ph, pl.g_nt[ph]); for (int t = 0; t < GMAX_T; ++t) printf("%d ", pl.g_len[ph][t]); printf("\n");
    for (int g = 0; g < GG; ++g) for (int t = 0; t < GMAX_T; ++t) {
      GrpTask tk = pl.gt[ph][g][t]; if (tk.a < 0) continue;
      if (t >= pl.g_nt[ph] || tk.n > pl.g_len[ph][t]) bad++;
      printf("  lane %d task %d: (%d,%d) n=%d off=%d\n", g, t, tk.a, tk.b, tk.n, tk.off);
      blk[tk.a][tk.b]++;
      int ra = cdim(P::ckind(tk.a)), rb = cdim(P::ckind(tk.b));
      if ((ph < 2) != (ra == 6) || ((ph % 2) == 0) != (rb == 6)) bad++, printf("shape\n");
      if (roff<P>(tk.a) < roff<P>(tk.b)) bad++;
      if (tk.off + tk.n > GMAX_POOL) bad++;
      std::set<int> js; for (int s = 0; s < tk.n; ++s) js.insert(pl.pool[tk.off + s]);
      for (int j = 0; j < D; ++j) { bool want = col_sign<P>(tk.a, j) && col_sign<P>(tk.b, j); if (want != (js.count(j) > 0)) bad++, printf("task joint set\n"); }
    }
  }
  for (int a = 0; a < NC; ++a) for (int b = 0; b < NC; ++b) {
    if (roff<P>(a) < roff<P>(b)) continue;
    bool nz = false; for (int j = 0; j < D; ++j) nz |= col_sign<P>(a, j) && col_sign<P>(b, j);
    if (a == b && grp_com_like<P>(a)) nz = false;  // dq-partition sum
    if (blk[a][b] != (nz ? 1 : 0)) bad++, printf("block (%d,%d) %d\n", a, b, blk[a][b]);
  }
  // refinement tasks: each constraint once with its column set
  int rs[NC] = {0};
  for (int ph = 0; ph < 2; ++ph) for (int g = 0; g < GG; ++g) for (int t = 0; t < GMAX_T; ++t) {
    GrpTask tk = pl.rt[ph][g][t]; if (tk.a < 0) continue; rs[tk.a]++;
    if (t >= pl.r_nt[ph] || tk.n > pl.r_len[ph][t]) bad++;
    std::set<int> js; for (int s = 0; s < tk.n; ++s) js.insert(pl.pool[tk.off + s]);
    for (int j = 0; j < D; ++j) if ((col_sign<P>(tk.a, j) != 0) != (js.count(j) > 0)) bad++;
  }
  for (int c = 0; c < NC; ++c) if (rs[c] != (grp_pose_like<P>(c) ? 1 : 0)) bad++, printf("refinement %d\n", c);
  // A mask: every entry written by a task is in the mask, every masked entry written
  {
    bool w[32][32] = {{false}};
    for (int ph = 0; ph < 4; ++ph) for (int g = 0; g < GG; ++g) for (int t = 0; t < GMAX_T; ++t) {
      GrpTask tk = pl.gt[ph][g][t]; if (tk.a < 0) continue;
      for (int i = 0; i < cdim(P::ckind(tk.a)); ++i) for (int k = 0; k < cdim(P::ckind(tk.b)); ++k) {
        int ii = roff<P>(tk.a) + i, kk = roff<P>(tk.b) + k; if (ii >= kk) w[ii][kk] = true; }
    }
    for (int c = 0; c < NC; ++c) if (grp_com_like<P>(c)) { int r0 = roff<P>(c); w[r0][r0] = w[r0 + 1][r0] = w[r0 + 1][r0 + 1] = true; }
    int nm = 0;
    for (int i = 0; i < K; ++i) for (int b = 0; b <= i; ++b) { bool m = (pl.amask[i] >> b) & 1; nm += m; if (m && !w[i][b]) bad++, printf("masked unwritten %d %d\n", i, b); }
    printf(" amask entries %d of %d\n", nm, K * (K + 1) / 2);
  }
  // The compile-time pattern of L (blocks the kernel skips): a Cholesky in
  // double of J J^T + lambda I, J random on its structural nonzeros, has an
  // exact zero wherever the pattern has one, and the pattern is no wider than
  // the factor (every entry it keeps is nonzero in this factor).
  {
    unsigned long long x = 0x9E3779B97F4A7C15ull;
    auto rnd = [&]() { x ^= x << 13; x ^= x >> 7; x ^= x << 17; return (double)(x >> 11) / 9007199254740992.0 - 0.5; };
    double J[32][64] = {{0}}, A[32][32] = {{0}}, Lm[32][32] = {{0}};
    for (int i = 0; i < K; ++i) for (int j = 0; j < D; ++j) if (jnz<P>(i, j)) J[i][j] = rnd();
    for (int i = 0; i < K; ++i) for (int b = 0; b < K; ++b) { double t = 0; for (int j = 0; j < D; ++j) t += J[i][j] * J[b][j]; A[i][b] = t + (i == b ? 1e-6 : 0.0); }
    for (int k = 0; k < K; ++k) {
      double d = A[k][k]; for (int j = 0; j < k; ++j) d -= Lm[k][j] * Lm[k][j];
      Lm[k][k] = std::sqrt(d);
      for (int i = k + 1; i < K; ++i) { double t = A[i][k]; for (int j = 0; j < k; ++j) t -= Lm[i][j] * Lm[k][j]; Lm[i][k] = t / Lm[k][k]; }
    }
    int zeros = 0;
    for (int i = 0; i < K; ++i) for (int b = 0; b <= i; ++b) {
      const bool nzp = (l_row_pattern<P>(i) >> b) & 1u;
      if (!nzp && Lm[i][b] != 0.0) bad++, printf("L[%d][%d] = %g outside the pattern\n", i, b, Lm[i][b]);
      if (nzp && Lm[i][b] == 0.0) bad++, printf("L[%d][%d] kept by the pattern but zero\n", i, b);
      zeros += !nzp;
    }
    printf(" L pattern: %d structural zeros of %d\n", zeros, K * (K + 1) / 2);
  }
  // L columns
  for (int i = 0; i < K; ++i) if (pl.lcol[i] != lcol_base<K>(i)) bad++;
  if (lcol_base<K>(K) > (int)(sizeof(GrpState<P>) )) bad++;
  printf(" sizes: GrpState %zu B, Eval %zu B, A %d, Lc %d floats, NJ %d, shared %zu B, smem(W=2) %zu B, args %zu B\n",
         sizeof(GrpState<P>), sizeof(typename GrpState<P>::Eval), GrpState<P>::K2, GrpState<P>::LC, NJ,
         sizeof(GrpShared<P>), group_smem_bytes<P>(2), sizeof(GroupArgs<P>));
  printf(" offsets: J %zu (mod8 %zu), u %zu (mod16 %zu), s.y %zu s.dq %zu, tables %zu\n", offsetof(GrpState<P>, J), offsetof(GrpState<P>, J) % 8, offsetof(GrpState<P>, u), offsetof(GrpState<P>, u) % 16,
         offsetof(typename GrpState<P>::Solve, y), offsetof(typename GrpState<P>::Solve, dq), sizeof(GrpTables<P>));
  printf(" %s: %d problems\n", P::name, bad);
  return bad;
}
int main() { return check<ProbHumanoid36>() + check<ProbHumanoid36Hull>(); }
