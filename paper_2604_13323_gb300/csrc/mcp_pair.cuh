// Two lanes per configuration for the dual arm: the persistent FP32
// projection with lane h of each pair (h = lane & 1) running chain h of the
// tree, for problem classes made of two copies of one serial chain coupled by
// the relative pose of their end frames (Eq. 2, T_err = T_ref^-1 T_a^-1 T_b).
//
// Per Newton step (Alg. 2 getDescentStep, stacked inner form):
//   * each lane runs FK of its own chain (half of the tree) and the two end
//     frames are exchanged by shuffles;
//   * both lanes evaluate the same residual from the same frames, so every
//     exit decision is taken identically by the two lanes of a pair;
//   * each lane builds its chain's 6 x 7 block of J (columns of chain 0 enter
//     with -1, those of chain 1 with +1) and its partial Gram B B^T; the two
//     partials are summed by one shuffle each (a + b = b + a exactly, so both
//     lanes hold the same A);
//   * both lanes factor A and solve; dq of each chain = s B^T y, one
//     refinement step with J dq summed over the pair.
// A configuration that leaves the loop is accepted in FP64 exactly as by the
// thread-per-configuration kernel (accept_one: 32 configurations per warp;
// a failed acceptance with steps left returns to the FP32 loop).
//
// Against one thread per configuration this halves the registers and the
// straight-line code of FK, Jacobian and Gram per lane (more warps resident,
// less instruction-cache pressure) and repeats the 6 x 6 residual and solve
// in both lanes.  The autotuner times both and keeps the faster.
#pragma once

#include "mcp_kernels.cuh"

namespace mcp {

// rows of one chain in a model: X[j] = model X[j0 + j], fX[0] = model fX[f0]
template <typename T>
struct ChainModel {
  const T (*X)[12];
  const T (*fX)[12];
};

// one chain of ProbDual14Rel: the 7-DoF DH arm with its end frame
struct ProbDual14Chain : ProbArm7Pose {
  static constexpr const char *name = "dual14_chain";
};

template <class P>
struct PairOf {
  static constexpr bool ok = false;
  using C = P;
};
template <>
struct PairOf<ProbDual14Rel> {
  static constexpr bool ok = true;
  using C = ProbDual14Chain;
};

// The pair layout holds only if P is chain C twice (chain h = joints h H ..
// h H + H - 1, end frame h) under one relative-pose constraint a = 0, b = 1.
template <class P, class C>
constexpr bool pair_layout_matches() {
  constexpr int H = C::D;
  if (P::D != 2 * H || P::NF != 2 || C::NF != 1 || P::NC != 1) return false;
  if (P::ckind(0) != K_REL || P::cfa(0) != 0 || P::cfb(0) != 1) return false;
  for (int j = 0; j < P::D; ++j) {
    const int h = j / H, jc = j % H;
    const int pc = C::parent(jc);
    if (P::parent(j) != (pc < 0 ? -1 : pc + h * H)) return false;
    if (P::jtype(j) != C::jtype(jc) || P::xrot(j) != C::xrot(jc) || P::xtmask(j) != C::xtmask(jc)) return false;
  }
  for (int h = 0; h < 2; ++h)
    if (P::frame_link(h) != C::frame_link(0) + h * H || P::frot(h) != C::frot(0) || P::ftmask(h) != C::ftmask(0))
      return false;
  return true;
}
static_assert(pair_layout_matches<ProbDual14Rel, ProbDual14Chain>(), "dual arm is not two copies of its chain");

// One FP32 Newton step of the configuration held by this lane's pair; q is
// this lane's chain.  pm names the two lanes of the pair.  Returns true when
// the configuration leaves the FP32 loop (the same value in both lanes).
template <class P, class A>
__device__ __forceinline__ bool pair_iter_f32(const A &a, int h, unsigned pm, float (&q)[PairOf<P>::C::D], int &it,
                                              uint32_t &fl) {
  using C = typename PairOf<P>::C;
  constexpr int H = C::D, K = 6;
  const OpsF32 ops{a.tab};
  Kin<C, float> k;
  const ChainModel<float> cm{a.m.X + H * h, a.m.fX + h};
  fk<C, true>(ops, cm, q, k);
  // both end frames in both lanes: kk.f*[0] = chain 0's, kk.f*[1] = chain 1's
  float mine[12], other[12];
#pragma unroll
  for (int i = 0; i < 9; ++i) mine[i] = k.fR[0][i];
  mine[9] = k.fp[0].x;
  mine[10] = k.fp[0].y;
  mine[11] = k.fp[0].z;
#pragma unroll
  for (int i = 0; i < 12; ++i) other[i] = __shfl_xor_sync(pm, mine[i], 1);
  Kin<P, float> kk;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    kk.fR[0][i] = h ? other[i] : mine[i];
    kk.fR[1][i] = h ? mine[i] : other[i];
  }
  kk.fp[0] = h ? V3<float>{other[9], other[10], other[11]} : V3<float>{mine[9], mine[10], mine[11]};
  kk.fp[1] = h ? V3<float>{mine[9], mine[10], mine[11]} : V3<float>{other[9], other[10], other[11]};
  float F[K];
  Eval<P, float> e;
  float qfull[P::D];  // read by configuration-space constraints only (none here)
#pragma unroll
  for (int j = 0; j < P::D; ++j) qfull[j] = 0.f;
  residual<P, OpsF32, float, true>(a.m, qfull, kk, F, e);
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
  // this chain's block B of J (J_h = s B, s = -1 for chain a, +1 for chain b)
  float B[K][H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    const V3<float> vt = mulv(e.G[0], cross(k.z[j], sub(e.x[0], k.p[j])));
    const V3<float> w = jl_inv_apply(e.phi[0], e.beta[0], mulv(e.G[0], k.z[j]));
    B[0][j] = vt.x;
    B[1][j] = vt.y;
    B[2][j] = vt.z;
    B[3][j] = w.x;
    B[4][j] = w.y;
    B[5][j] = w.z;
  }
  const float s = h ? 1.f : -1.f;
  // A = B_0 B_0^T + B_1 B_1^T + lambda I
  float Am[K * (K + 1) / 2], inv[K];
#pragma unroll
  for (int r = 0; r < K; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      float t = 0.f;
#pragma unroll
      for (int j = 0; j < H; ++j) t = fmaf(B[r][j], B[c][j], t);
      Am[tri(r, c)] = t;
    }
#pragma unroll
  for (int i = 0; i < K * (K + 1) / 2; ++i) Am[i] += __shfl_xor_sync(pm, Am[i], 1);
#pragma unroll
  for (int i = 0; i < K; ++i) Am[tri(i, i)] += a.lambda;
  const float piv = cholesky_factor<K, OpsF32>(Am, inv);
  if (!(piv >= a.pivot)) {  // also catches NaN: finish this configuration in FP64
    fl |= FL_INT_NEEDS_F64;
    return true;
  }
  float y[K];
#pragma unroll
  for (int i = 0; i < K; ++i) y[i] = F[i];
  cholesky_subst<K>(Am, inv, y);
  float dq[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    float t = 0.f;
#pragma unroll
    for (int r = 0; r < K; ++r) t = fmaf(B[r][j], y[r], t);
    dq[j] = s * t;
  }
  // refinement: r = F - J dq - lambda y with J dq = sum over the pair of s B dq_h
  float rr[K];
#pragma unroll
  for (int r = 0; r < K; ++r) {
    float t = 0.f;
#pragma unroll
    for (int j = 0; j < H; ++j) t = fmaf(B[r][j], dq[j], t);
    rr[r] = s * t;
  }
#pragma unroll
  for (int r = 0; r < K; ++r) {
    const float u = rr[r] + __shfl_xor_sync(pm, rr[r], 1);
    rr[r] = fmaf(-a.lambda, y[r], F[r] - u);
  }
  cholesky_subst<K>(Am, inv, rr);
#pragma unroll
  for (int r = 0; r < K; ++r) y[r] += rr[r];
  float s2h = 0.f;
#pragma unroll
  for (int j = 0; j < H; ++j) {
    float t = 0.f;
#pragma unroll
    for (int r = 0; r < K; ++r) t = fmaf(B[r][j], y[r], t);
    dq[j] = s * t * a.alpha;
    s2h = fmaf(dq[j], dq[j], s2h);
  }
  const float s2 = s2h + __shfl_xor_sync(pm, s2h, 1);
  if (a.max_step2 > 0.f && s2 > a.max_step2) {
    fl |= FL_DIV;
    return true;
  }
#pragma unroll
  for (int j = 0; j < H; ++j) q[j] -= dq[j];
  ++it;
  fl &= ~FL_INT_FORCE;
  if (!(s2 <= FLT_MAX)) {
    fl |= FL_NONFINITE;
    return true;
  }
  return false;
}

constexpr int PAIR_REGS = 96;  // 5 blocks of 128 threads per SM (20 warps); 128 registers: 16 warps, 5 % slower
template <int TPB>
__host__ __device__ constexpr int pair_min_blocks() {
  return 65536 / (TPB * PAIR_REGS) > 0 ? 65536 / (TPB * PAIR_REGS) : 1;
}

// The persistent loop of k_project_f32 with pairs as slots (16 per warp):
// warp-local work queue, refill of idle pairs, parked configurations accepted
// in FP64 32 at a time.
template <class P, class Src, int TPB, bool CHK>
__global__ void __launch_bounds__(TPB, (pair_min_blocks<TPB>())) k_project_pair(const __grid_constant__ ProjArgs<P, Src> a) {
  using C = typename PairOf<P>::C;
  constexpr int H = C::D;
  constexpr int W = TPB / 32;
  constexpr unsigned EVEN = 0x55555555u;  // one lane (h = 0) per pair
  __shared__ long long s_item[W][64];
  __shared__ uint32_t s_meta[W][64];
  __shared__ long long s_ritem[W][RETRY_CAP];
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
  const int h = lane & 1;
  const unsigned pm = 3u << (lane & 30);
  const unsigned before = (1u << (lane & 30)) - 1u;  // lanes of the pairs before this one
  const long long total = a.src.clamp_total(a.total);
  int pend = 0;              // warp-uniform count of parked configurations
  int nret = 0;              // warp-uniform count of configurations to retry in FP32
  long long qn = 0, qe = 0;  // warp-local queue [qn, qe)
  bool more = true;
  bool act = false;  // the same in both lanes of a pair
  long long item = 0;
  int it = 0;
  uint32_t fl = 0;
  float q[H];
#pragma unroll
  for (int j = 0; j < H; ++j) q[j] = 0.f;

  while (true) {
    // (1) refill idle pairs: retries first, then new work
    const unsigned idle = __ballot_sync(FULL, !act) & EVEN;
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
      const int rank_all = __popc(idle & before);
      if (!act) {
        if (rank_all < from_r) {  // one more FP32 step from the parked iterate
          const int pos = nret - 1 - rank_all;
          item = s_ritem[wib][pos];
          const uint32_t meta = s_rmeta[wib][pos];
          it = static_cast<int>(meta & 0xffu);
          fl = ((meta >> 8) & ~(FL_INT_FP32CONV | FL_INT_NEEDS_F64)) | FL_INT_FORCE;
          act = true;
#pragma unroll
          for (int j = 0; j < H; ++j) q[j] = MCP_CHK(item, a.ld_out) ? a.q_out[(H * h + j) * a.ld_out + item] : 0.f;
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
            a.src.template load_part<H>(item, H * h, q);
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
    // (2) one FP32 Newton step per active pair
    bool done = false;
    if (act) done = pair_iter_f32<P>(a, h, pm, q, it, fl);
    // (3) park finished configurations
    const unsigned fin = __ballot_sync(FULL, done) & EVEN;
    if (fin != 0u) {
      if (done) {
        if (MCP_CHK(item, a.ld_out)) {
#pragma unroll
          for (int j = 0; j < H; ++j) a.q_out[(H * h + j) * a.ld_out + item] = q[j];
        }
        if (h == 0) {
          const int pos = pend + __popc(fin & before);
          s_item[wib][pos] = item;
          s_meta[wib][pos] = static_cast<uint32_t>(it) | (fl << 8);
        }
        act = false;
      }
      pend += __popc(fin);
      __syncwarp();
    }
    const bool drained = !__any_sync(FULL, act) && qn >= qe && !more && nret == 0;
    // (4) FP64 acceptance, one configuration per lane; a failed acceptance
    // with steps left goes back to the FP32 loop
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
        if constexpr (CHK) {  // the collision check of the accepted output, one configuration per lane
          if (!retry) {
            float qc[P::D];
            const bool okc = MCP_CHK(it_item, a.ld_out);
#pragma unroll
            for (int j = 0; j < P::D; ++j) qc[j] = okc ? a.q_out[j * a.ld_out + it_item] : 0.f;
            uint32_t tests = 0;
            const bool hit = check_one_f32<P>(a.chk->m, a.chk->st, s_pair, a.n_obs, s_box, a.n_box, a.tab, qc, tests);
            if (okc) a.hit[it_item] = hit ? 1 : 0;
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

template <class P, class Src, int TPB, bool CHK>
cudaError_t launch_pair_tpb(const HostModel &hm, const ProjCall &c, const Src &src) {
  ProjArgs<P, Src> a{};
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
  const long long warps_needed = (2 * c.total + 31) / 32;
  long long blocks = static_cast<long long>(hm.sm_count) * c.tune.blocks_per_sm;
  const long long max_useful = (warps_needed + (TPB / 32) - 1) / (TPB / 32);
  if (blocks > max_useful) blocks = max_useful;
  if (blocks < 1) blocks = 1;
  k_project_pair<P, Src, TPB, CHK><<<static_cast<unsigned>(blocks), TPB, smem, c.stream>>>(a);
  return cudaGetLastError();
}

template <class P, class Src, bool CHK>
cudaError_t launch_pair(const HostModel &hm, const ProjCall &c, const Src &src) {
  switch (c.tune.tpb) {
    case 64: return launch_pair_tpb<P, Src, 64, CHK>(hm, c, src);
    case 256: return launch_pair_tpb<P, Src, 256, CHK>(hm, c, src);
    default: return launch_pair_tpb<P, Src, 128, CHK>(hm, c, src);
  }
}

}  // namespace mcp
