// Batched ParallelConstrainedExtend (Algorithm 2): one group of lanes per
// extension (8 lanes for up to 8 particles, else the warp), its lanes playing
// the paper's SIMD lanes.  Lanes hold the n particles around
// q_steer, then the n points interpolated between q_s and q_proj, then the
// bisection midpoints; every point is projected by the per-thread FP32 Newton
// loop with FP64 acceptance and collision-checked against the obstacles in
// shared memory, and the early exits of the algorithm are warp votes.
//
// The particles and points are projected each with its own exit.  The
// lockstep exits of Alg. 2 then read: the particle projection succeeds if some
// particle converges no later than the first step that exceeds MaxDistance
// (the convergence test of an iteration precedes its step); the winner is the
// particle that converged after the fewest steps, the lowest lane on ties.
#pragma once

#include "mcp_kernels.cuh"

namespace mcp {

constexpr int EXT_MAXPTS = 128;  // points of the validated chain, both ends included
enum : int {
  EXT_OK = 0, EXT_DEGENERATE = 1, EXT_NO_PROJECTION = 2, EXT_PROJ_COLLISION = 3, EXT_TOO_FAR = 4,
  EXT_INTERP_FAIL = 5, EXT_GAP = 6, EXT_INTERP_COLLISION = 7, EXT_RESOLUTION = 8
};

template <class P>
struct ExtArgs {
  ModelT<float> m;
  const ModelT<double> *__restrict__ m64;
  const double2 *__restrict__ tab;
  const CheckData *chk;
  const float *obs;
  const float *box;
  int n_obs;
  int n_box;
  const float *q_s;
  const float *q_t;
  long long ld;
  const float *eps;
  long long ld_eps;
  float *q_proj;
  uint8_t *status;
  int32_t *n_points;
  int32_t *winner;
  int32_t *steps;  // optional: Newton steps of all projections of the extension
  float *scratch;  // validated chains: 2 x EXT_MAXPTS x D floats per resident group
  long long n_ext;
  unsigned long long *counter;
  int n;
  int max_depth;
  float r;
  float delta;
  int cap;
  float tol2;
  float lambda;
  float max_step2;
  float pivot;
  double tol2_64;
  double lambda64;
  float alpha;
};

// FP64 acceptance of one FP32 iterate held in registers (accept_one without
// the global outputs).  Out of line: it runs once per projection, and kept
// apart from the Newton loop it does not dilute the loop's instruction stream.
// Returns true (nothing changed) when the FP32 test was too optimistic and
// steps remain: the caller takes one more FP32 step and asks again.
template <class P, class A>
__device__ __noinline__ bool accept_regs(const A &a, float (&q)[P::D], int &it, uint32_t &fl) {
  constexpr int D = P::D;
  double r2 = residual2_f64<P>(OpsF64Split{a.tab}, *a.m64, q);
  if ((fl & FL_INT_FP32CONV) && !(r2 < a.tol2_64) && r2 <= DBL_MAX && it < a.cap) return true;
  if (fl & (FL_INT_FP32CONV | FL_INT_NEEDS_F64)) {
    const bool was_conv = (fl & FL_INT_FP32CONV) != 0;
    fl &= ~(FL_INT_FP32CONV | FL_INT_NEEDS_F64);
    if (r2 < a.tol2_64) {
      fl |= FL_CONV;
    } else {
      float qf[D];
      double qd[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        qf[j] = q[j];
        qd[j] = static_cast<double>(q[j]);
      }
      finish_f64<P, FORM_STACKED>(a, qf, qd, &it, &fl, r2, was_conv);
#pragma unroll
      for (int j = 0; j < D; ++j) q[j] = qf[j];
    }
  }
  return false;
}

// Projects the point of every active lane (warp-convergent: all lanes call
// it).  Out of line: the extension calls it at three places and one copy keeps
// the kernel within the instruction cache.
template <class P, class A>
__device__ __noinline__ void project_lanes(const A &a, float (&q)[P::D], bool active, int &it, uint32_t &fl) {
  it = 0;
  fl = 0;
  bool done = !active;
  bool final_ = !active;  // accepted (or inactive)
  while (true) {
    while (__any_sync(FULL, !done)) {
      if (!done) done = newton_iter_f32<P>(a, q, it, fl);
    }
    bool again = false;
    if (!final_) {
      again = accept_regs<P>(a, q, it, fl);
      final_ = !again;
    }
    if (!__any_sync(FULL, again)) break;
    if (again) {  // one more FP32 step before the next test
      fl = (fl & ~(FL_INT_FP32CONV | FL_INT_NEEDS_F64)) | FL_INT_FORCE;
      done = false;
    }
  }
}

// Collision verdict of one lane's configuration, out of line (called at three places).
template <class P>
__device__ __noinline__ bool collides_lane(const CheckData *chk, const float4 *s_pair, int n_obs, const float *s_box,
                                           int n_box, const double2 *tab, const float (&q)[P::D]) {
  uint32_t t = 0;  // the flat broad phase: this kernel is bound by instruction fetch
  return check_one_f32<P, false>(chk->m, chk->st, s_pair, n_obs, s_box, n_box, tab, q, t);
}

template <int D>
__device__ __forceinline__ float pt_dist(const float *x, const float *y) {
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < D; ++j) s = fmaf(x[j] - y[j], x[j] - y[j], s);
  return sqrtf(s);
}
template <int D>
__device__ __forceinline__ float pt_dist_r(const float *x, const float (&y)[D]) {
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < D; ++j) s = fmaf(x[j] - y[j], x[j] - y[j], s);
  return sqrtf(s);
}

// One extension per group of G lanes (G = 8: four extensions per warp, for
// n <= 8 particles; G = 32: one per warp).  The groups of a warp step through
// Alg. 2's stages together, because the projection is warp-collective; a
// group whose extension has ended idles through the remaining stages.  Votes,
// minima and broadcasts are taken over the group's lanes.
template <class P, int W, int G>
__global__ void __launch_bounds__(W * 32) k_extend(const __grid_constant__ ExtArgs<P> a) {
  constexpr int D = P::D;
  constexpr int NG = 32 / G;
  static_assert(G == 8 || G == 16 || G == 32, "groups of 8, 16 or 32 lanes");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4 *s_pair = reinterpret_cast<float4 *>(smem_raw);
  const float *s_box = stage_obstacles(a.obs, a.n_obs, a.box, a.n_box, s_pair);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane % G, gbase = grp * G;
  const unsigned gbits = G == 32 ? FULL : ((1u << G) - 1u);
  const unsigned lt = (1u << gl) - 1u;  // group lanes below this one
  // this group's two chain buffers (global scratch, one pair per resident group)
  const size_t slot = (static_cast<size_t>(blockIdx.x) * W + wib) * NG + grp;
  float *chain = a.scratch + slot * 2 * EXT_MAXPTS * D;  // [EXT_MAXPTS][D]
  float *next = chain + EXT_MAXPTS * D;
  auto collides = [&](const float (&q)[D]) -> bool {
    return collides_lane<P>(a.chk, s_pair, a.n_obs, s_box, a.n_box, a.tab, q);
  };
  // group votes (every lane of the warp must call them)
  auto gballot = [&](bool v) -> unsigned { return (__ballot_sync(FULL, v) >> gbase) & gbits; };
  auto gmin = [&](unsigned v) -> unsigned {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(FULL, v, o));
    return v;
  };
  auto gsum = [&](int v) -> int {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
  };
  while (true) {
    unsigned long long e = 0;
    if (lane == 0) e = atomicAdd(a.counter, static_cast<unsigned long long>(NG));
    e = __shfl_sync(FULL, e, 0);
    if (static_cast<long long>(e) >= a.n_ext) break;
    const long long x = static_cast<long long>(e) + grp;
    const bool valid = x < a.n_ext;
    float qs[D], qt[D], qp[D], v[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      qs[j] = valid ? a.q_s[j * a.ld + x] : 0.f;
      qt[j] = valid ? a.q_t[j * a.ld + x] : 0.f;
      qp[j] = qs[j];
    }
    int status = EXT_OK, npts = 0, win = -1;
    int work = 0;  // this lane's Newton steps
    float len2 = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) len2 = fmaf(qt[j] - qs[j], qt[j] - qs[j], len2);
    const float len = sqrtf(len2);
    const bool act = gl < a.n;  // particle / interpolated-point lane
    int it = 0;
    uint32_t fl = 0;
    bool alive = valid;
    if (valid && !(len > 0.f)) {
      status = EXT_DEGENERATE;
      alive = false;
    }
    // steer and the particles around it along the extension direction
    const float dist = fminf(len, a.r);
    float p[D];
    {
      const float ep = (alive && act) ? a.eps[gl * a.ld_eps + x] : 0.f;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        v[j] = alive ? (qt[j] - qs[j]) / len : 0.f;
        p[j] = fmaf(ep, v[j], fmaf(dist, v[j], qs[j]));
      }
    }
    project_lanes<P>(a, p, alive && act, it, fl);
    if (alive && act) work += it;
    {
      constexpr unsigned BIG = 0xffffffffu;
      const unsigned c = (alive && act && (fl & FL_CONV)) ? static_cast<unsigned>(it) : BIG;
      const unsigned dv = (alive && act && (fl & FL_DIV)) ? static_cast<unsigned>(it) : BIG;
      const unsigned minc = gmin(c), mindv = gmin(dv);
      const unsigned wb = gballot(c == minc);
      const int w = wb ? __ffs(static_cast<int>(wb)) - 1 : 0;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const float t = __shfl_sync(FULL, p[j], gbase + w);
        if (alive && minc != BIG && !(mindv < minc)) qp[j] = t;
      }
      if (alive && (minc == BIG || mindv < minc)) {
        status = EXT_NO_PROJECTION;
        alive = false;
      } else if (alive) {
        win = w;
        npts = 1;
      }
    }
    // the projected point: collision (one lane per group), the 2 dist exit
    {
      const bool pc = (alive && gl == 0) ? collides(qp) : false;
      const bool hit = gballot(pc) != 0u;
      float d2 = 0.f;
#pragma unroll
      for (int j = 0; j < D; ++j) d2 = fmaf(qp[j] - qs[j], qp[j] - qs[j], d2);
      if (alive && hit) {
        status = EXT_PROJ_COLLISION;
        alive = false;
      } else if (alive && sqrtf(d2) > 2.f * dist) {
        status = EXT_TOO_FAR;
        alive = false;
      }
    }
    // n points between q_s and q_proj (lane k of the group: t = (k + 1) / (n + 1))
    float xq[D];
    {
      const float tk = static_cast<float>(gl + 1) / static_cast<float>(a.n + 1);
#pragma unroll
      for (int j = 0; j < D; ++j) xq[j] = fmaf(tk, qp[j] - qs[j], qs[j]);
    }
    project_lanes<P>(a, xq, alive && act, it, fl);
    if (alive && act) work += it;
    const bool unconv = gballot(act && !(fl & FL_CONV)) != 0u;  // every lane votes
    if (alive && unconv) {
      status = EXT_INTERP_FAIL;
      alive = false;
    }
    if (alive) npts += a.n;
    // the chain q_s, x_1 .. x_n, q_proj
    if (alive) {
      if (gl == 0) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
          chain[j] = qs[j];
          chain[(a.n + 1) * D + j] = qp[j];
        }
      }
      if (act) {
#pragma unroll
        for (int j = 0; j < D; ++j) chain[(gl + 1) * D + j] = xq[j];
      }
    }
    __syncwarp();
    int m = a.n + 2;
    {
      bool gap = false;
      for (int k0 = 0; k0 < m - 1; k0 += G) {  // m is the same for every group here
        const int k = k0 + gl;
        gap |= gballot(alive && k < m - 1 && pt_dist<D>(chain + k * D, chain + (k + 1) * D) > a.r / a.n) != 0u;
      }
      if (alive && gap) {
        status = EXT_GAP;
        alive = false;
      }
      const bool cx = (alive && act) ? collides(xq) : false;
      const bool xhit = gballot(cx) != 0u;  // every lane votes
      if (alive && xhit) {
        status = EXT_INTERP_COLLISION;
        alive = false;
      }
    }
    // bisect every gap above the resolution, level by level
    bool bis = alive;
    for (int level = 0; __any_sync(FULL, bis); ++level) {
      int mmax = bis ? m : 0;  // chunk loops run over the longest chain of the warp
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mmax = max(mmax, __shfl_xor_sync(FULL, mmax, o));
      int wide = 0;
      for (int k0 = 0; k0 < mmax - 1; k0 += G) {
        const int k = k0 + gl;
        const bool w = bis && k < m - 1 && pt_dist<D>(chain + k * D, chain + (k + 1) * D) > a.delta;
        wide += __popc(gballot(w));
      }
      if (bis && wide == 0) {
        bis = false;  // resolved: the extension is valid
      } else if (bis && (level >= a.max_depth || m + wide > EXT_MAXPTS)) {
        status = EXT_RESOLUTION;
        bis = false;
      }
      if (!__any_sync(FULL, bis)) break;
      int base_w = 0;
      bool failed = false;
      for (int k0 = 0; k0 < mmax - 1; k0 += G) {
        const int k = k0 + gl;
        const bool in = bis && !failed && k < m - 1;
        const float g = in ? pt_dist<D>(chain + k * D, chain + (k + 1) * D) : 0.f;
        const bool w = in && g > a.delta;
        const unsigned bal = gballot(w);
        const int pos = k + base_w + __popc(bal & lt);
        float mq[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const float lo = in ? chain[k * D + j] : 0.f;
          const float hi = in ? chain[(k + 1) * D + j] : 0.f;
          if (in) next[pos * D + j] = lo;
          mq[j] = 0.5f * (lo + hi);
        }
        project_lanes<P>(a, mq, w, it, fl);
        if (w) work += it;
        int code = 0;
        if (w) {
          if (!(fl & FL_CONV)) code = EXT_INTERP_FAIL;
          else if (pt_dist_r<D>(chain + k * D, mq) > g || pt_dist_r<D>(chain + (k + 1) * D, mq) > g)
            code = EXT_GAP;
          else if (collides(mq)) code = EXT_INTERP_COLLISION;
          if (code == 0) {
#pragma unroll
            for (int j = 0; j < D; ++j) next[(pos + 1) * D + j] = mq[j];
          }
        }
        const unsigned fb = gballot(code != 0);
        const int fl_lane = fb ? __ffs(static_cast<int>(fb)) - 1 : 0;
        const int fcode = __shfl_sync(FULL, code, gbase + fl_lane);
        if (bis && !failed && fb) {
          status = fcode;
          npts += base_w + __popc(bal & ((1u << fl_lane) - 1u));
          failed = true;
        }
        base_w += __popc(bal);
      }
      if (bis && failed) bis = false;
      if (bis) {
        npts += wide;
        if (gl == 0) {
#pragma unroll
          for (int j = 0; j < D; ++j) next[(m - 1 + wide) * D + j] = chain[(m - 1) * D + j];
        }
        m += wide;
        float *t = chain;
        chain = next;
        next = t;
      }
      __syncwarp();
    }
    const int work_all = gsum(work);
    if (valid && gl == 0) {
#pragma unroll
      for (int j = 0; j < D; ++j) a.q_proj[j * a.ld + x] = qp[j];
      a.status[x] = static_cast<uint8_t>(status);
      a.n_points[x] = npts;
      a.winner[x] = win;
      if (a.steps) a.steps[x] = work_all;
    }
    __syncwarp();
  }
}

template <class P, int G>
cudaError_t launch_extend_g(const HostModel &hm, const ExtCall &c, ExtArgs<P> &a, int *launches) {
  constexpr int W = 2;
  auto kern = k_extend<P, W, G>;
  const size_t smem = obs_smem_bytes(hm.n_obs, hm.n_box);
  cudaError_t err = cudaSuccess;
  if (smem > 48 * 1024) err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  constexpr int NG = 32 / G;
  long long blocks = static_cast<long long>(hm.sm_count) * per_sm;
  const long long need = (c.n_ext + W * NG - 1) / (W * NG);
  if (blocks > need) blocks = need;
  // two chains of EXT_MAXPTS points per resident group
  const size_t floats = static_cast<size_t>(blocks) * W * NG * 2 * EXT_MAXPTS * P::D;
  if (!c.scratch) return cudaErrorInvalidValue;
  if (c.scratch->floats < floats) {
    cudaFree(c.scratch->ptr);
    c.scratch->ptr = nullptr;
    c.scratch->floats = 0;
    err = dev_malloc(&c.scratch->ptr, floats * sizeof(float), "extend chain scratch");
    if (err != cudaSuccess) return err;
    c.scratch->floats = floats;
  }
  a.scratch = c.scratch->ptr;
  err = cudaMemsetAsync(c.counter, 0, sizeof(unsigned long long), c.stream);
  if (err != cudaSuccess) return err;
  kern<<<static_cast<unsigned>(blocks), W * 32, smem, c.stream>>>(a);
  *launches += 1;
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_extend_impl(const HostModel &hm, const ExtCall &c, int *launches) {
  if (c.n_ext <= 0) return cudaSuccess;
  ExtArgs<P> a;
  a.m = hm.m32;
  a.m64 = hm.d_m64;
  a.tab = hm.d_tab;
  a.chk = hm.d_chk;
  a.obs = reinterpret_cast<const float *>(hm.d_obs32);
  a.box = hm.d_box32;
  a.n_obs = hm.n_obs;
  a.n_box = hm.n_box;
  a.q_s = c.q_s;
  a.q_t = c.q_t;
  a.ld = c.ld;
  a.eps = c.eps;
  a.ld_eps = c.ld_eps;
  a.q_proj = c.q_proj;
  a.status = c.status;
  a.n_points = c.n_points;
  a.winner = c.winner;
  a.steps = c.steps;
  a.n_ext = c.n_ext;
  a.counter = c.counter;
  a.n = c.n;
  a.max_depth = c.max_depth;
  a.r = static_cast<float>(c.r);
  a.delta = static_cast<float>(c.delta);
  a.cap = c.cap;
  a.tol2 = static_cast<float>(c.tol * c.tol);
  a.lambda = static_cast<float>(c.lambda);
  a.max_step2 = c.max_step > 0 ? static_cast<float>(c.max_step * c.max_step) : 0.f;
  a.pivot = static_cast<float>(c.pivot);
  a.tol2_64 = c.tol * c.tol;
  a.lambda64 = c.lambda;
  a.alpha = static_cast<float>(c.alpha);
  a.scratch = nullptr;
  // lanes per extension: the particles rounded up to a group of 8 or the warp
  return c.n <= 8 ? launch_extend_g<P, 8>(hm, c, a, launches) : launch_extend_g<P, 32>(hm, c, a, launches);
}

}  // namespace mcp

#define MCP_INSTANTIATE_EXTEND(P)                                                                \
  namespace mcp {                                                                                \
  template <>                                                                                    \
  cudaError_t launch_extend<P>(const HostModel &hm, const ExtCall &c, int *launches) {            \
    return launch_extend_impl<P>(hm, c, launches);                                               \
  }                                                                                              \
  }
