// C ABI of libmcproj.so (declared in include/mcproj.h): context, model
// loading, binding of a loaded robot/constraint stack to a compiled problem
// class, and the batched entry points.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/mcproj.h"
#include "mcp_device.cuh"
#include "mcp_internal.h"
#include "mcp_problems.cuh"

using namespace mcp;

namespace mcp {
static std::atomic<long long> g_allocs{0};

// Readers of the per-module error words of the bounds-check mode (each
// module of a -DMCP_CHECK_BOUNDS build registers one when it is loaded).
static std::vector<unsigned int (*)(bool)> &bounds_readers() {
  static std::vector<unsigned int (*)(bool)> r;
  return r;
}
void register_bounds_reader(unsigned int (*reader)(bool)) { bounds_readers().push_back(reader); }
unsigned int bounds_error_of_all_modules(bool reset) {
  unsigned int first = 0;
  for (auto *rd : bounds_readers()) {
    const unsigned int v = rd(reset);
    if (v && !first) first = v;
  }
  return first;
}

cudaError_t dev_malloc(void **p, size_t bytes, const char *label) {
  const char *f = std::getenv("MCP_TEST_FAIL_ALLOC");
  if (f && *f && std::strstr(label, f)) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_allocs.fetch_add(1, std::memory_order_relaxed);
  return e;
}
}  // namespace mcp

// ---------------------------------------------------------------------------
// Problem-class registry
// ---------------------------------------------------------------------------
namespace {

struct ClassDesc {
  const char *name;
  int D, NF, NC;
  int parent[MAXJ], jtype[MAXJ], xrot[MAXJ], xtmask[MAXJ];
  int flink[MAXF], frot[MAXF], ftmask[MAXF];
  int ckind[MAXC], cfa[MAXC], cfb[MAXC];
  bool project;  // projection / VJP compiled for this class
  bool pair;     // the FP32 projection also runs one lane per chain (threads per configuration 2)
  cudaError_t (*project_fn)(const HostModel &, const ProjCall &, int *);
  cudaError_t (*check_fn)(const HostModel &, const CheckCall &, int *);
  cudaError_t (*vjp_fn)(const HostModel &, const VjpCall &, int *);
  cudaError_t (*extend_fn)(const HostModel &, const ExtCall &, int *);
};

template <class P>
ClassDesc describe(bool project) {
  ClassDesc d{};
  d.name = P::name;
  d.D = P::D;
  d.NF = P::NF;
  d.NC = P::NC;
  for (int j = 0; j < P::D; ++j) {
    d.parent[j] = P::parent(j);
    d.jtype[j] = P::jtype(j);
    d.xrot[j] = P::xrot(j);
    d.xtmask[j] = P::xtmask(j);
  }
  for (int f = 0; f < P::NF; ++f) {
    d.flink[f] = P::frame_link(f);
    d.frot[f] = P::frot(f);
    d.ftmask[f] = P::ftmask(f);
  }
  for (int c = 0; c < P::NC; ++c) {
    d.ckind[c] = P::ckind(c);
    d.cfa[c] = P::cfa(c);
    d.cfb[c] = P::cfb(c);
  }
  d.project = project;
  d.pair = has_pair_kernel<P>();
  d.project_fn = &launch_project<P>;
  d.check_fn = &launch_check<P>;
  d.vjp_fn = &launch_vjp<P>;
  d.extend_fn = &launch_extend<P>;
  return d;
}

const std::vector<ClassDesc> &registry() {
  static const std::vector<ClassDesc> r = {
      describe<ProbSphere3>(true),   describe<ProbPoint3Planes4>(true), describe<ProbArm7Axis>(true),
      describe<ProbArm7Pose>(true),
      describe<ProbArm7Tray>(true),  describe<ProbArm7Peg>(true),   describe<ProbArm7Tsr>(true),
      describe<ProbDual14Rel>(true), describe<ProbDual14Rod>(true), describe<ProbHumanoid36>(true),
      describe<ProbHumanoid36Hull>(true)};
  return r;
}

// Signed-permutation code of a rotation given exactly (entries 0 / +-1), or XR_GENERIC.
int rot_code(const double *X) {
  int code = 0;
  for (int k = 0; k < 3; ++k) {
    int row = -1;
    for (int r = 0; r < 3; ++r) {
      const double v = X[r * 4 + k];
      if (v == 0.0) continue;
      if ((v != 1.0 && v != -1.0) || row >= 0) return XR_GENERIC;
      row = r;
    }
    if (row < 0) return XR_GENERIC;
    code |= row << (2 * k);
    if (X[row * 4 + k] < 0) code |= 1 << (6 + k);
  }
  return code;
}

int trans_mask(const double *X) {
  return (X[3] != 0.0 ? 1 : 0) | (X[7] != 0.0 ? 2 : 0) | (X[11] != 0.0 ? 4 : 0);
}

struct RobotHost {
  int nj = 0, ns = 0, nf = 0;
  std::vector<int> parent, type, sphere_link, frame_link;
  std::vector<double> X, lower, upper, mass, com, sphere, frame_X;
};

struct ConsHost {
  int kind, fa, fb;
  double P[12], Q[12], target[3], B[12];
  bool has_ref;
  std::vector<double> q_ref;
};

// Setup-kernel input (resolution of q_ref references, subtree masses).
struct ResolveIn {
  int nj, nf, nc;
  int parent[MAXJ], type[MAXJ], flink[MAXF];
  double X[MAXJ][12], fX[MAXF][12], mass[MAXJ];
  int kind[MAXC], fa[MAXC], fb[MAXC], has_ref[MAXC];
  double P[MAXC][12], Q[MAXC][12], tgt[MAXC][3], B[MAXC][12];
  double qref[MAXC][MAXJ];
};
struct ResolveOut {
  double P[MAXC][12], Q[MAXC][12], tgt[MAXC][3], B[MAXC][12];
  double Pinv[MAXC][12], Qinv[MAXC][12];
  double msub[MAXJ];
  double inv_mass;
};

}  // namespace

// ---------------------------------------------------------------------------
// Setup kernels (FP64, run once per load)
// ---------------------------------------------------------------------------
__global__ void k_sincos_table(double2 *tab) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < 256) {  // (sin, cos)(2 pi k / 256)
    double s, c;
    sincospi(static_cast<double>(k) / 128.0, &s, &c);
    tab[k] = make_double2(s, c);
  } else if (k < SPLIT_TAB_OFF + 2 * SPLIT_TAB_HALF + 1) {  // (sin, cos)(m / 512), m = -2048..2048
    double s, c;
    sincos(static_cast<double>(k - SPLIT_TAB_OFF - SPLIT_TAB_HALF) / 512.0, &s, &c);
    tab[k] = make_double2(s, c);
  }
}

__device__ void tf_mul64(const double *A, const double *B, double *C) {
  double o[12];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = A[r * 4] * B[c] + A[r * 4 + 1] * B[4 + c] + A[r * 4 + 2] * B[8 + c];
      if (c == 3) s += A[r * 4 + 3];
      o[r * 4 + c] = s;
    }
  for (int i = 0; i < 12; ++i) C[i] = o[i];
}
__device__ void tf_inv64(const double *A, double *B) {
  double o[12];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) o[r * 4 + c] = A[c * 4 + r];
    o[r * 4 + 3] = -(A[r] * A[3] + A[4 + r] * A[7] + A[8 + r] * A[11]);
  }
  for (int i = 0; i < 12; ++i) B[i] = o[i];
}

// One thread: FK at each constraint's q_ref (runtime topology), references,
// inverses, subtree masses.
__global__ void k_resolve(const __grid_constant__ ResolveIn in, ResolveOut *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double T[MAXJ][12], Tf[MAXF][12];
  for (int c = 0; c < in.nc; ++c) {
    for (int i = 0; i < 12; ++i) {
      out->P[c][i] = in.P[c][i];
      out->Q[c][i] = in.Q[c][i];
    }
    for (int i = 0; i < 3; ++i) out->tgt[c][i] = in.tgt[c][i];
    for (int i = 0; i < 12; ++i) out->B[c][i] = in.B[c][i];
    if (in.has_ref[c]) {
      for (int j = 0; j < in.nj; ++j) {
        double pre[12], M[12];
        if (in.parent[j] < 0) {
          for (int i = 0; i < 12; ++i) pre[i] = in.X[j][i];
        } else {
          tf_mul64(T[in.parent[j]], in.X[j], pre);
        }
        for (int i = 0; i < 12; ++i) M[i] = 0.0;
        M[0] = M[5] = M[10] = 1.0;
        const double qj = in.qref[c][j];
        if (in.type[j] == REV) {
          double s, cc;
          sincos(qj, &s, &cc);
          M[0] = cc; M[1] = -s; M[4] = s; M[5] = cc;
        } else {
          M[11] = qj;
        }
        tf_mul64(pre, M, T[j]);
      }
      for (int f = 0; f < in.nf; ++f) {
        if (in.flink[f] < 0) {
          for (int i = 0; i < 12; ++i) Tf[f][i] = in.fX[f][i];
        } else {
          tf_mul64(T[in.flink[f]], in.fX[f], Tf[f]);
        }
      }
      const int a = in.fa[c], b = in.fb[c];
      if (in.kind[c] == K_POSE || in.kind[c] == K_PBND) {
        double Qi[12];
        tf_inv64(in.Q[c], Qi);
        tf_mul64(Tf[a], Qi, out->P[c]);
      } else if (in.kind[c] == K_PLANE || in.kind[c] == K_LINE) {
        // the plane / line keeps its orientation and passes through frame a
        out->P[c][3] = Tf[a][3];
        out->P[c][7] = Tf[a][7];
        out->P[c][11] = Tf[a][11];
      } else if (in.kind[c] == K_DIST) {
        const double dx = Tf[b][3] - Tf[a][3], dy = Tf[b][7] - Tf[a][7], dz = Tf[b][11] - Tf[a][11];
        out->tgt[c][0] = sqrt(dx * dx + dy * dy + dz * dz);
      } else if (in.kind[c] == K_REL) {
        double Ai[12];
        tf_inv64(Tf[a], Ai);
        tf_mul64(Ai, Tf[b], out->P[c]);
      } else if (in.kind[c] == K_COM) {
        out->tgt[c][0] = 0.5 * (Tf[a][3] + Tf[b][3]);
        out->tgt[c][1] = 0.5 * (Tf[a][7] + Tf[b][7]);
      } else if (in.kind[c] == K_HULL) {
        // the support polygon: the xy box around frames a and b grown by the margin tgt[1]
        const double mg = in.tgt[c][1];
        const double x0 = fmin(Tf[a][3], Tf[b][3]) - mg, x1 = fmax(Tf[a][3], Tf[b][3]) + mg;
        const double y0 = fmin(Tf[a][7], Tf[b][7]) - mg, y1 = fmax(Tf[a][7], Tf[b][7]) + mg;
        const double v[8] = {x0, y0, x1, y0, x1, y1, x0, y1};
        for (int i = 0; i < 8; ++i) out->B[c][i] = v[i];
        out->tgt[c][0] = 4.0;
      }
    }
    tf_inv64(out->P[c], out->Pinv[c]);
    tf_inv64(out->Q[c], out->Qinv[c]);
  }
  double M = 0.0;
  for (int j = in.nj - 1; j >= 0; --j) out->msub[j] = in.mass[j];
  for (int j = in.nj - 1; j >= 0; --j) {
    if (in.parent[j] >= 0) out->msub[in.parent[j]] += out->msub[j];
    M += in.mass[j];
  }
  out->inv_mass = M > 0.0 ? 1.0 / M : 0.0;
}

// Obstacle preparation (one block): centroid of the obstacle centres (FP64),
// then per obstacle sphere the FP32 records of the expanded overlap test in
// the shifted frame: (-2c, |c|^2 - r^2), (-2r, 0, 0, 0); after them, one
// record of the same form per chunk of OBS_CHUNK consecutive obstacles: a
// sphere around the chunk (centre the mean of its centres, radius the largest
// |c_o - c| + r_o plus 1e-4 m, which keeps the FP32 test of the chunk
// conservative); boxes shifted.
__global__ void k_prep_obstacles(const double *obs, int n_obs, const double *box, int n_box, float *obs32,
                                 float *box32, double *origin) {
  __shared__ double part[3][256];
  const int t = threadIdx.x;
  double sx = 0.0, sy = 0.0, sz = 0.0;
  for (int o = t; o < n_obs; o += blockDim.x) {
    sx += obs[4 * o];
    sy += obs[4 * o + 1];
    sz += obs[4 * o + 2];
  }
  if (n_obs == 0)
    for (int b = t; b < n_box; b += blockDim.x) {
      sx += 0.5 * (box[6 * b] + box[6 * b + 3]);
      sy += 0.5 * (box[6 * b + 1] + box[6 * b + 4]);
      sz += 0.5 * (box[6 * b + 2] + box[6 * b + 5]);
    }
  part[0][t] = sx;
  part[1][t] = sy;
  part[2][t] = sz;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (t < w)
      for (int c = 0; c < 3; ++c) part[c][t] += part[c][t + w];
    __syncthreads();
  }
  const int cnt = n_obs > 0 ? n_obs : n_box;
  const double ox = cnt ? part[0][0] / cnt : 0.0, oy = cnt ? part[1][0] / cnt : 0.0, oz = cnt ? part[2][0] / cnt : 0.0;
  if (t == 0) {
    origin[0] = ox;
    origin[1] = oy;
    origin[2] = oz;
  }
  for (int o = t; o < n_obs; o += blockDim.x) {
    const double cx = obs[4 * o] - ox, cy = obs[4 * o + 1] - oy, cz = obs[4 * o + 2] - oz, r = obs[4 * o + 3];
    obs32[8 * o + 0] = static_cast<float>(-2.0 * cx);
    obs32[8 * o + 1] = static_cast<float>(-2.0 * cy);
    obs32[8 * o + 2] = static_cast<float>(-2.0 * cz);
    obs32[8 * o + 3] = static_cast<float>(cx * cx + cy * cy + cz * cz - r * r);
    obs32[8 * o + 4] = static_cast<float>(-2.0 * r);
    obs32[8 * o + 5] = 0.f;
    obs32[8 * o + 6] = 0.f;
    obs32[8 * o + 7] = 0.f;
  }
  for (int k = t; k < obs_chunks(n_obs); k += blockDim.x) {
    const int o0 = k * OBS_CHUNK, o1 = o0 + OBS_CHUNK < n_obs ? o0 + OBS_CHUNK : n_obs;
    double mx = 0.0, my = 0.0, mz = 0.0;
    for (int o = o0; o < o1; ++o) {
      mx += obs[4 * o] - ox;
      my += obs[4 * o + 1] - oy;
      mz += obs[4 * o + 2] - oz;
    }
    mx /= (o1 - o0);
    my /= (o1 - o0);
    mz /= (o1 - o0);
    double rad = 0.0;
    for (int o = o0; o < o1; ++o) {
      const double dx = obs[4 * o] - ox - mx, dy = obs[4 * o + 1] - oy - my, dz = obs[4 * o + 2] - oz - mz;
      const double e = sqrt(dx * dx + dy * dy + dz * dz) + obs[4 * o + 3];
      rad = e > rad ? e : rad;
    }
    rad += 1e-4;
    float *rec = obs32 + 8 * (n_obs + k);
    rec[0] = static_cast<float>(-2.0 * mx);
    rec[1] = static_cast<float>(-2.0 * my);
    rec[2] = static_cast<float>(-2.0 * mz);
    rec[3] = static_cast<float>(mx * mx + my * my + mz * mz - rad * rad);
    rec[4] = static_cast<float>(-2.0 * rad);
    rec[5] = rec[6] = rec[7] = 0.f;
  }
  for (int b = t; b < n_box; b += blockDim.x) {
    box32[6 * b + 0] = static_cast<float>(box[6 * b + 0] - ox);
    box32[6 * b + 1] = static_cast<float>(box[6 * b + 1] - oy);
    box32[6 * b + 2] = static_cast<float>(box[6 * b + 2] - oz);
    box32[6 * b + 3] = static_cast<float>(box[6 * b + 3] - ox);
    box32[6 * b + 4] = static_cast<float>(box[6 * b + 4] - oy);
    box32[6 * b + 5] = static_cast<float>(box[6 * b + 5] - oz);
  }
}

// Bounding sphere of each link's spheres (local coordinates), one thread per
// group: centre = mean of the sphere centres, radius = max(|c_s - centre| +
// r_s) + 1e-4 m, so that an FP32 overlap test against it is conservative.
// Group g < nj is link g; group MAXJ holds the world-fixed spheres.
__global__ void k_link_bounds(const SphereTable<double> *st, int nj, double *out /* (MAXJ + 1) * 4 */) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g > MAXJ) return;
  const int l = (g == MAXJ) ? -1 : g;
  double *o = out + 4 * g;
  o[0] = o[1] = o[2] = o[3] = 0.0;
  if (l >= nj) return;
  const int s0 = st->off[l + 1], e = st->off[l + 2];
  if (s0 >= e) return;
  double cx = 0.0, cy = 0.0, cz = 0.0;
  for (int s = s0; s < e; ++s) {
    cx += st->s[s][0];
    cy += st->s[s][1];
    cz += st->s[s][2];
  }
  cx /= (e - s0);
  cy /= (e - s0);
  cz /= (e - s0);
  double r = 0.0;
  for (int s = s0; s < e; ++s) {
    const double dx = st->s[s][0] - cx, dy = st->s[s][1] - cy, dz = st->s[s][2] - cz;
    const double v = sqrt(dx * dx + dy * dy + dz * dz) + st->s[s][3];
    r = v > r ? v : r;
  }
  o[0] = cx;
  o[1] = cy;
  o[2] = cz;
  o[3] = r + 1e-4;
}

// Exclusive prefix sum of segment lengths into off[0..n]; one block.
__global__ void k_scan_lengths(const int32_t *len, long long n, long long *off) {
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const long long per = (n + blockDim.x - 1) / blockDim.x;
  const long long b = t * per, e = (b + per < n) ? b + per : n;
  long long s = 0;
  for (long long i = b; i < e; ++i) s += len[i] > 0 ? len[i] : 0;
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    long long acc = 0;
    for (int i = 0; i < static_cast<int>(blockDim.x); ++i) {
      const long long v = part[i];
      part[i] = acc;
      acc += v;
    }
    off[n] = acc;
  }
  __syncthreads();
  long long acc = part[t];
  for (long long i = b; i < e; ++i) {
    off[i] = acc;
    acc += len[i] > 0 ? len[i] : 0;
  }
}

// Path length and its gradient (thread per waypoint / per path).
// One thread per waypoint: d/dq_i of |q_i - q_{i-1}| + |q_{i+1} - q_i|, in two
// passes over the joints (the norms, then the output; the second pass re-reads
// the same waypoints from L1) so that nothing is held in runtime-indexed arrays.
__global__ void k_path_grad(const float *Q, long long ld, long long n_paths, int n_way, int d, float *grad) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_paths * n_way) return;
  const int w = static_cast<int>(i % n_way);
  const bool has_p = w > 0, has_n = w + 1 < n_way;
  float np2 = 0.f, nn2 = 0.f;
  for (int j = 0; j < d; ++j) {
    const float qi = Q[j * ld + i];
    const float ep = has_p ? qi - Q[j * ld + i - 1] : 0.f;
    const float en = has_n ? Q[j * ld + i + 1] - qi : 0.f;
    np2 = fmaf(ep, ep, np2);
    nn2 = fmaf(en, en, nn2);
  }
  const float ip = np2 > 0.f ? rsqrtf(np2) : 0.f;
  const float in = nn2 > 0.f ? rsqrtf(nn2) : 0.f;
  for (int j = 0; j < d; ++j) {
    const float qi = Q[j * ld + i];
    const float ep = has_p ? qi - Q[j * ld + i - 1] : 0.f;
    const float en = has_n ? Q[j * ld + i + 1] - qi : 0.f;
    grad[j * ld + i] = ep * ip - en * in;
  }
}

__global__ void k_path_step(float *Q, const float *D, long long ld, long long n_paths, int n_way, int d, float eta,
                            float max_step) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_paths * n_way) return;
  const int w = static_cast<int>(i % n_way);
  if (w == 0 || w == n_way - 1) return;  // endpoints stay fixed
  float m = 0.f;
  for (int j = 0; j < d; ++j) m = fmaxf(m, fabsf(eta * D[j * ld + i]));
  const float sc = (max_step > 0.f && m > max_step) ? max_step / m : 1.f;
  for (int j = 0; j < d; ++j) Q[j * ld + i] = fmaf(-sc * eta, D[j * ld + i], Q[j * ld + i]);
}

// One warp per path: lane l sums the lengths of segments l, l + 32, ... and
// the warp adds the partial sums in a fixed order (deterministic).
__global__ void k_path_length(const float *Q, long long ld, long long n_paths, int n_way, int d, float *length) {
  const long long p = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= n_paths) return;  // whole warps leave together
  float L = 0.f;
  for (int w = lane; w + 1 < n_way; w += 32) {
    const long long i = p * n_way + w;
    float n2 = 0.f;
    for (int j = 0; j < d; ++j) {
      const float e = Q[j * ld + i + 1] - Q[j * ld + i];
      n2 = fmaf(e, e, n2);
    }
    L += sqrtf(n2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) L += __shfl_xor_sync(0xffffffffu, L, o);
  if (lane == 0) length[p] = L;
}

// Arithmetic-throughput probe: every thread advances 8 independent FMA
// chains x <- x a + b for `iters` rounds (a < 1, so the chains stay bounded).
// The final sum is written only if it is negative, which it never is; the
// compiler cannot know that, so no chain is removed.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T *out, long long iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = static_cast<T>(threadIdx.x + c);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  if (s < T(0)) out[0] = s;
}

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct mcp_ctx {
  int device = 0;
  std::string err;
  std::string fail_cuda;  // test hook: CUDA calls whose label contains it report an error (MCP_TEST_FAIL_CUDA)
  bool robot_loaded = false, cons_loaded = false, obs_loaded = false;
  RobotHost robot;
  std::vector<ConsHost> cons;
  HostModel hm;
  int robot_class = -1;  // class whose robot part matches (collision check)
  int prob_class = -1;   // class whose robot and constraints match (projection, VJP)
  ModelT<double> *d_m64 = nullptr;
  CheckData *d_chk = nullptr;
  double2 *d_tab = nullptr;
  float4 *d_obs32 = nullptr;
  double *d_obs64 = nullptr;
  float *d_box32 = nullptr;
  double *d_box64 = nullptr;
  double *d_origin = nullptr;
  double origin[3] = {0.0, 0.0, 0.0};
  unsigned long long *d_counter = nullptr;
  ScratchBuf ext_scratch;  // extend_batch: the validated chains
  long long *d_seg_off = nullptr;
  long long seg_cap = 0;
  ResolveOut *d_resolve = nullptr;
  Tuning tune;
  bool tuned = false;
  int64_t launches = 0;
  uint64_t version = 0;  // bumped by every load: invalidates captured graphs
  // captured segment-projection graph and the arguments it was captured with
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t seg_exec = nullptr;
  std::vector<unsigned char> seg_key;
  int seg_graph_launches = 0;  // kernels inside the captured graph
};

namespace {

mcp_status fail(mcp_ctx *c, mcp_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

mcp_status cuda_fail(mcp_ctx *c, cudaError_t e, const char *what) {
  if (e == cudaErrorNotSupported) {
    cudaGetLastError();
    return fail(c, MCP_ERR_UNSUPPORTED, "%s: not compiled for this problem class / precision / source", what);
  }
  return fail(c, e == cudaErrorMemoryAllocation ? MCP_ERR_OOM : MCP_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

// Host-side failure injection for tests: with the environment variable
// MCP_TEST_FAIL_CUDA set when the context was created, a CUDA call of this
// context whose label contains its text reports cudaErrorLaunchFailure after
// it has run (nothing on the device fails; the context stays usable).
cudaError_t injected(const mcp_ctx *ctx, cudaError_t e, const char *what) {
  if (e != cudaSuccess || !ctx || ctx->fail_cuda.empty()) return e;
  return std::strstr(what, ctx->fail_cuda.c_str()) ? cudaErrorLaunchFailure : cudaSuccess;
}

#define MCP_CUDA(call, what)                                    \
  do {                                                          \
    cudaError_t e_ = injected(ctx, (call), what);               \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what);     \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool robot_matches(const ClassDesc &d, const RobotHost &r) {
  if (d.D != r.nj || d.NF != r.nf) return false;
  for (int j = 0; j < r.nj; ++j) {
    if (d.parent[j] != r.parent[j] || d.jtype[j] != r.type[j]) return false;
    const int code = rot_code(&r.X[12 * j]);
    if (d.xrot[j] != XR_GENERIC && d.xrot[j] != code) return false;
    if (d.parent[j] >= 0 && (trans_mask(&r.X[12 * j]) & ~d.xtmask[j])) return false;
  }
  for (int f = 0; f < r.nf; ++f) {
    if (d.flink[f] != r.frame_link[f]) return false;
    const int code = rot_code(&r.frame_X[12 * f]);
    if (d.frot[f] != XR_GENERIC && d.frot[f] != code) return false;
    if (trans_mask(&r.frame_X[12 * f]) & ~d.ftmask[f]) return false;
  }
  return true;
}

bool cons_match(const ClassDesc &d, const std::vector<ConsHost> &c) {
  if (d.NC != static_cast<int>(c.size())) return false;
  for (int i = 0; i < d.NC; ++i) {
    if (d.ckind[i] != c[i].kind) return false;
    const bool uses_a = c[i].kind != K_SPHERE && c[i].kind != K_COM;
    const bool uses_b = c[i].kind == K_REL || c[i].kind == K_DIST;
    if (uses_a && d.cfa[i] != c[i].fa) return false;
    if (uses_b && d.cfb[i] != c[i].fb) return false;
  }
  return true;
}

void bind_classes(mcp_ctx *ctx) {
  ctx->robot_class = -1;
  ctx->prob_class = -1;
  const auto &reg = registry();
  for (int i = 0; i < static_cast<int>(reg.size()); ++i) {
    if (!ctx->robot_loaded || !robot_matches(reg[i], ctx->robot)) continue;
    if (ctx->robot_class < 0) ctx->robot_class = i;
    if (ctx->cons_loaded && reg[i].project && cons_match(reg[i], ctx->cons)) {
      ctx->prob_class = i;
      ctx->robot_class = i;
      break;
    }
  }
}

template <typename T>
void fill_sphere_table(const RobotHost &r, SphereTable<T> &st) {
  std::memset(&st, 0, sizeof(st));
  int n = 0;
  for (int l = -1; l < r.nj; ++l) {
    st.off[l + 1] = static_cast<int16_t>(n);
    for (int s = 0; s < r.ns; ++s) {
      if (r.sphere_link[s] != l) continue;
      for (int i = 0; i < 4; ++i) st.s[n][i] = static_cast<T>(r.sphere[4 * s + i]);
      ++n;
    }
  }
  st.off[r.nj + 1] = static_cast<int16_t>(n);
  for (int l = r.nj + 2; l < MAXJ + 2; ++l) st.off[l] = static_cast<int16_t>(n);
}

// Joint limits in precision T rounded outwards-in: lower up, upper down.  For a
// value q exactly representable in T, q < lower_T iff q < lower and
// q > upper_T iff q > upper, so limit flags of FP32 iterates need no FP64.
template <typename T>
T bound_up(double v) {
  T t = static_cast<T>(v);
  if (static_cast<double>(t) < v) t = std::nextafter(t, std::numeric_limits<T>::infinity());
  return t;
}
template <typename T>
T bound_down(double v) {
  T t = static_cast<T>(v);
  if (static_cast<double>(t) > v) t = std::nextafter(t, -std::numeric_limits<T>::infinity());
  return t;
}

template <typename T>
void fill_robot_model(const RobotHost &r, ModelT<T> &m) {
  std::memset(&m, 0, sizeof(m));
  for (int j = 0; j < r.nj; ++j) {
    for (int i = 0; i < 12; ++i) m.X[j][i] = static_cast<T>(r.X[12 * j + i]);
    m.mass[j] = static_cast<T>(r.mass[j]);
    for (int i = 0; i < 3; ++i) m.com[j][i] = static_cast<T>(r.com[3 * j + i]);
    m.lower[j] = bound_up<T>(r.lower[j]);
    m.upper[j] = bound_down<T>(r.upper[j]);
  }
  for (int f = 0; f < r.nf; ++f)
    for (int i = 0; i < 12; ++i) m.fX[f][i] = static_cast<T>(r.frame_X[12 * f + i]);
}

template <typename T>
void fill_constraints(const ResolveOut &ro, const std::vector<ConsHost> &cons, int nj, ModelT<T> &m) {
  const int nc = static_cast<int>(cons.size());
  for (int c = 0; c < nc; ++c) {
    for (int i = 0; i < 12; ++i) {
      m.cPinv[c][i] = static_cast<T>(ro.Pinv[c][i]);
      m.cQinv[c][i] = static_cast<T>(ro.Qinv[c][i]);
      m.cB[c][i] = static_cast<T>(ro.B[c][i]);
    }
    for (int i = 0; i < 3; ++i) m.ctgt[c][i] = static_cast<T>(ro.tgt[c][i]);
  }
  for (int j = 0; j < nj; ++j) m.msub[j] = static_cast<T>(ro.msub[j]);
  m.inv_mass = static_cast<T>(ro.inv_mass);
}

// The collision-frame copy of the FP32 model: root offsets minus the obstacle
// origin; also uploaded (with the sphere table) for the fused check.
mcp_status update_shifted(mcp_ctx *ctx) {
  ctx->hm.m32_shifted = ctx->hm.m32;
  for (int j = 0; j < ctx->robot.nj; ++j) {
    if (ctx->robot.parent[j] >= 0) continue;
    for (int r = 0; r < 3; ++r)
      ctx->hm.m32_shifted.X[j][r * 4 + 3] = static_cast<float>(ctx->robot.X[12 * j + r * 4 + 3] - ctx->origin[r]);
  }
  for (int r = 0; r < 3; ++r) ctx->hm.m32_shifted.shift[r] = static_cast<float>(ctx->origin[r]);
  if (!ctx->d_chk) {
    cudaError_t e = dev_malloc(&ctx->d_chk, sizeof(CheckData), "check data");
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc check data");
    ctx->hm.d_chk = ctx->d_chk;
  }
  CheckData *h = new (std::nothrow) CheckData;
  if (!h) return fail(ctx, MCP_ERR_OOM, "host allocation failed");
  h->m = ctx->hm.m32_shifted;
  h->st = ctx->hm.st32;
  cudaError_t e = cudaMemcpy(ctx->d_chk, h, sizeof(CheckData), cudaMemcpyHostToDevice);
  delete h;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "check data copy");
  return MCP_OK;
}

mcp_status check_batch_ptr(mcp_ctx *ctx, const void *p, const char *name) {
  if (!p) return fail(ctx, MCP_ERR_ARG, "%s is NULL", name);
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, MCP_ERR_ARG, "%s is not a CUDA-visible pointer", name);
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(ctx, MCP_ERR_ARG, "%s must be device memory", name);
  return MCP_OK;
}

mcp_status ensure_resolved(mcp_ctx *ctx) {
  // (re)build FP32/FP64 models from the loaded robot and constraints
  DeviceGuard g(ctx->device);
  ResolveIn *in = new (std::nothrow) ResolveIn;
  if (!in) return fail(ctx, MCP_ERR_OOM, "host allocation failed");
  std::memset(in, 0, sizeof(ResolveIn));
  const RobotHost &r = ctx->robot;
  in->nj = r.nj;
  in->nf = r.nf;
  in->nc = static_cast<int>(ctx->cons.size());
  for (int j = 0; j < r.nj; ++j) {
    in->parent[j] = r.parent[j];
    in->type[j] = r.type[j];
    in->mass[j] = r.mass[j];
    for (int i = 0; i < 12; ++i) in->X[j][i] = r.X[12 * j + i];
  }
  for (int f = 0; f < r.nf; ++f) {
    in->flink[f] = r.frame_link[f];
    for (int i = 0; i < 12; ++i) in->fX[f][i] = r.frame_X[12 * f + i];
  }
  for (int c = 0; c < in->nc; ++c) {
    const ConsHost &ch = ctx->cons[c];
    in->kind[c] = ch.kind;
    in->fa[c] = ch.fa;
    in->fb[c] = ch.fb;
    in->has_ref[c] = ch.has_ref ? 1 : 0;
    for (int i = 0; i < 12; ++i) {
      in->P[c][i] = ch.P[i];
      in->Q[c][i] = ch.Q[i];
    }
    for (int i = 0; i < 3; ++i) in->tgt[c][i] = ch.target[i];
    for (int i = 0; i < 12; ++i) in->B[c][i] = ch.B[i];
    if (ch.has_ref)
      for (int j = 0; j < r.nj; ++j) in->qref[c][j] = ch.q_ref[j];
  }
  if (!ctx->d_resolve) {
    cudaError_t e = dev_malloc(&ctx->d_resolve, sizeof(ResolveOut), "reference resolution");
    if (e != cudaSuccess) {
      delete in;
      return cuda_fail(ctx, e, "cudaMalloc");
    }
  }
  k_resolve<<<1, 32>>>(*in, ctx->d_resolve);
  ctx->launches += 1;
  delete in;
  ResolveOut ro;
  MCP_CUDA(cudaGetLastError(), "resolve kernel launch");
  MCP_CUDA(cudaMemcpy(&ro, ctx->d_resolve, sizeof(ro), cudaMemcpyDeviceToHost), "resolve copy");
  for (int c = 0; c < static_cast<int>(ctx->cons.size()); ++c) {
    std::memcpy(ctx->cons[c].P, ro.P[c], sizeof(ro.P[c]));
    std::memcpy(ctx->cons[c].Q, ro.Q[c], sizeof(ro.Q[c]));
    std::memcpy(ctx->cons[c].target, ro.tgt[c], sizeof(ro.tgt[c]));
    std::memcpy(ctx->cons[c].B, ro.B[c], sizeof(ro.B[c]));
  }
  fill_robot_model(r, ctx->hm.m32);
  fill_robot_model(r, ctx->hm.m64);
  fill_constraints(ro, ctx->cons, r.nj, ctx->hm.m32);
  fill_constraints(ro, ctx->cons, r.nj, ctx->hm.m64);
  fill_sphere_table(r, ctx->hm.st32);
  fill_sphere_table(r, ctx->hm.st64);
  {
    SphereTable<double> *d_st = nullptr;
    double *d_lb = nullptr;
    MCP_CUDA(dev_malloc(&d_st, sizeof(SphereTable<double>), "sphere table"), "cudaMalloc sphere table");
    cudaError_t e = dev_malloc(&d_lb, (MAXJ + 1) * 4 * sizeof(double), "link bounds");
    if (e == cudaSuccess) e = cudaMemcpy(d_st, &ctx->hm.st64, sizeof(SphereTable<double>), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      k_link_bounds<<<1, 64>>>(d_st, r.nj, d_lb);
      ctx->launches += 1;
      e = cudaGetLastError();
    }
    double lb[(MAXJ + 1) * 4];
    if (e == cudaSuccess) e = cudaMemcpy(lb, d_lb, sizeof(lb), cudaMemcpyDeviceToHost);
    cudaFree(d_st);
    cudaFree(d_lb);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "link bounds");
    for (int g = 0; g <= MAXJ; ++g)
      for (int c = 0; c < 4; ++c) {
        ctx->hm.st64.lb[g][c] = lb[4 * g + c];
        ctx->hm.st32.lb[g][c] = static_cast<float>(lb[4 * g + c]);
      }
  }
  MCP_CUDA(cudaMemcpy(ctx->d_m64, &ctx->hm.m64, sizeof(ModelT<double>), cudaMemcpyHostToDevice), "model copy");
  return update_shifted(ctx);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

mcp_status mcp_create(int device, mcp_ctx **out) {
  if (!out) return MCP_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return MCP_ERR_ARG;
  }
  mcp_ctx *ctx = new (std::nothrow) mcp_ctx;
  if (!ctx) return MCP_ERR_OOM;
  ctx->device = device;
  if (const char *f = std::getenv("MCP_TEST_FAIL_CUDA")) ctx->fail_cuda = f;
  DeviceGuard g(device);
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  ctx->hm.sm_count = sms;
  cudaError_t e = dev_malloc(&ctx->d_m64, sizeof(ModelT<double>), "context model");
  if (e == cudaSuccess) e = dev_malloc(&ctx->d_tab, (SPLIT_TAB_OFF + 2 * SPLIT_TAB_HALF + 1) * sizeof(double2), "context tables");
  if (e == cudaSuccess) e = dev_malloc(&ctx->d_counter, sizeof(unsigned long long), "context counter");
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    k_sincos_table<<<(SPLIT_TAB_OFF + 2 * SPLIT_TAB_HALF + 1 + 255) / 256, 256>>>(ctx->d_tab);
    ctx->launches += 1;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    mcp_destroy(ctx);
    return MCP_ERR_CUDA;
  }
  ctx->hm.d_m64 = ctx->d_m64;
  ctx->hm.d_tab = ctx->d_tab;
  *out = ctx;
  return MCP_OK;
}

void mcp_destroy(mcp_ctx *ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  cudaFree(ctx->d_m64);
  cudaFree(ctx->d_chk);
  cudaFree(ctx->d_tab);
  cudaFree(ctx->d_obs32);
  cudaFree(ctx->d_obs64);
  cudaFree(ctx->d_box32);
  cudaFree(ctx->d_box64);
  cudaFree(ctx->d_counter);
  cudaFree(ctx->ext_scratch.ptr);
  cudaFree(ctx->d_seg_off);
  cudaFree(ctx->d_resolve);
  cudaFree(ctx->d_origin);
  if (ctx->seg_exec) cudaGraphExecDestroy(ctx->seg_exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

const char *mcp_last_error(const mcp_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int64_t mcp_launch_count(const mcp_ctx *ctx) { return ctx ? ctx->launches : 0; }

int64_t mcp_alloc_count(void) { return g_allocs.load(std::memory_order_relaxed); }

mcp_status mcp_bounds_status(const mcp_ctx *ctx, int32_t *enabled, uint32_t *first_line, int32_t reset) {
  if (!ctx) return MCP_ERR_ARG;
#ifdef MCP_CHECK_BOUNDS
  DeviceGuard g(ctx->device);
  if (cudaDeviceSynchronize() != cudaSuccess) return MCP_ERR_CUDA;
  const unsigned int v = bounds_error_of_all_modules(reset != 0);
  if (enabled) *enabled = 1;
  if (first_line) *first_line = v;
#else
  (void)reset;
  if (enabled) *enabled = 0;
  if (first_line) *first_line = 0;
#endif
  return MCP_OK;
}

mcp_status mcp_load_robot(mcp_ctx *ctx, const mcp_robot_desc *rd) {
  if (!ctx) return MCP_ERR_ARG;
  if (!rd) return fail(ctx, MCP_ERR_ARG, "robot descriptor is NULL");
  const int nj = rd->n_joints;
  if (nj < 1 || nj > MCP_MAX_JOINTS) return fail(ctx, MCP_ERR_ARG, "n_joints %d outside [1, %d]", nj, MCP_MAX_JOINTS);
  if (rd->n_spheres < 0 || rd->n_spheres > MCP_MAX_SPHERES)
    return fail(ctx, MCP_ERR_ARG, "n_spheres %d outside [0, %d]", rd->n_spheres, MCP_MAX_SPHERES);
  if (rd->n_frames < 0 || rd->n_frames > MCP_MAX_FRAMES)
    return fail(ctx, MCP_ERR_ARG, "n_frames %d outside [0, %d]", rd->n_frames, MCP_MAX_FRAMES);
  if (!rd->parent || !rd->type || !rd->X || !rd->lower || !rd->upper)
    return fail(ctx, MCP_ERR_ARG, "robot arrays parent/type/X/lower/upper are required");
  if (rd->n_spheres > 0 && (!rd->sphere_link || !rd->sphere)) return fail(ctx, MCP_ERR_ARG, "sphere arrays missing");
  if (rd->n_frames > 0 && (!rd->frame_link || !rd->frame_X)) return fail(ctx, MCP_ERR_ARG, "frame arrays missing");
  RobotHost r;
  r.nj = nj;
  r.ns = rd->n_spheres;
  r.nf = rd->n_frames;
  for (int j = 0; j < nj; ++j) {
    if (rd->parent[j] < -1 || rd->parent[j] >= j)
      return fail(ctx, MCP_ERR_ARG, "parent[%d] = %d must be in [-1, %d)", j, rd->parent[j], j);
    if (rd->type[j] != REV && rd->type[j] != PRIS) return fail(ctx, MCP_ERR_ARG, "type[%d] = %d", j, rd->type[j]);
  }
  r.parent.assign(rd->parent, rd->parent + nj);
  r.type.assign(rd->type, rd->type + nj);
  r.X.assign(rd->X, rd->X + 12 * nj);
  r.lower.assign(rd->lower, rd->lower + nj);
  r.upper.assign(rd->upper, rd->upper + nj);
  if (rd->mass) r.mass.assign(rd->mass, rd->mass + nj);
  else r.mass.assign(nj, 0.0);
  if (rd->com) r.com.assign(rd->com, rd->com + 3 * nj);
  else r.com.assign(3 * nj, 0.0);
  for (int s = 0; s < r.ns; ++s)
    if (rd->sphere_link[s] < -1 || rd->sphere_link[s] >= nj)
      return fail(ctx, MCP_ERR_ARG, "sphere_link[%d] = %d out of range", s, rd->sphere_link[s]);
  for (int f = 0; f < r.nf; ++f)
    if (rd->frame_link[f] < -1 || rd->frame_link[f] >= nj)
      return fail(ctx, MCP_ERR_ARG, "frame_link[%d] = %d out of range", f, rd->frame_link[f]);
  if (r.ns) {
    r.sphere_link.assign(rd->sphere_link, rd->sphere_link + r.ns);
    r.sphere.assign(rd->sphere, rd->sphere + 4 * r.ns);
  }
  if (r.nf) {
    r.frame_link.assign(rd->frame_link, rd->frame_link + r.nf);
    r.frame_X.assign(rd->frame_X, rd->frame_X + 12 * r.nf);
  }
  ctx->robot = std::move(r);
  ctx->robot_loaded = true;
  ++ctx->version;
  ctx->cons.clear();
  ctx->cons_loaded = false;
  ctx->tuned = false;
  bind_classes(ctx);
  return ensure_resolved(ctx);
}

mcp_status mcp_load_constraints(mcp_ctx *ctx, const mcp_constraint_desc *cd, int32_t n) {
  if (!ctx) return MCP_ERR_ARG;
  if (!ctx->robot_loaded) return fail(ctx, MCP_ERR_STATE, "load the robot before the constraints");
  if (n < 0 || n > MCP_MAX_CONSTRAINTS) return fail(ctx, MCP_ERR_ARG, "n = %d outside [0, %d]", n, MCP_MAX_CONSTRAINTS);
  if (n > 0 && !cd) return fail(ctx, MCP_ERR_ARG, "constraint array is NULL");
  std::vector<ConsHost> cons;
  int k = 0;
  for (int i = 0; i < n; ++i) {
    const mcp_constraint_desc &c = cd[i];
    if (c.kind < MCP_C_SPHERE || c.kind > MCP_C_COM_HULL)
      return fail(ctx, MCP_ERR_ARG, "constraint %d: kind %d", i, c.kind);
    const bool com = c.kind == MCP_C_COM_XY || c.kind == MCP_C_COM_HULL;
    const bool uses_a = c.kind != MCP_C_SPHERE && (!com || c.q_ref);
    const bool uses_b = c.kind == MCP_C_REL_POSE || c.kind == MCP_C_DIST || (com && c.q_ref);
    if (uses_a && (c.frame_a < 0 || c.frame_a >= ctx->robot.nf))
      return fail(ctx, MCP_ERR_ARG, "constraint %d: frame_a %d out of range", i, c.frame_a);
    if (uses_b && (c.frame_b < 0 || c.frame_b >= ctx->robot.nf))
      return fail(ctx, MCP_ERR_ARG, "constraint %d: frame_b %d out of range", i, c.frame_b);
    ConsHost h;
    h.kind = c.kind;
    h.fa = c.frame_a;
    h.fb = c.frame_b;
    std::memcpy(h.P, c.P, sizeof(h.P));
    std::memcpy(h.Q, c.Q, sizeof(h.Q));
    std::memcpy(h.target, c.target, sizeof(h.target));
    std::memcpy(h.B, c.B, sizeof(h.B));
    if (c.kind == MCP_C_POSE_BOUNDED)
      for (int r = 0; r < 6; ++r)
        if (!(c.B[r] <= c.B[6 + r]))
          return fail(ctx, MCP_ERR_ARG, "constraint %d: bound %d has lower > upper or NaN", i, r);
    if (c.kind == MCP_C_COM_HULL && !c.q_ref && !(c.target[0] >= 3.0 && c.target[0] <= 6.0))
      return fail(ctx, MCP_ERR_ARG, "constraint %d: a support polygon has 3 to 6 vertices", i);
    h.has_ref = c.q_ref != nullptr;
    if (h.has_ref) h.q_ref.assign(c.q_ref, c.q_ref + ctx->robot.nj);
    k += cdim(c.kind);
    cons.push_back(std::move(h));
  }
  if (k > MCP_MAX_EQUATIONS) return fail(ctx, MCP_ERR_ARG, "%d equations > %d", k, MCP_MAX_EQUATIONS);
  ctx->cons = std::move(cons);
  ctx->cons_loaded = true;
  ++ctx->version;
  ctx->tuned = false;
  bind_classes(ctx);
  return ensure_resolved(ctx);
}

mcp_status mcp_get_constraint(const mcp_ctx *ctx, int32_t i, double *P, double *Q, double *target, double *B) {
  if (!ctx || i < 0 || i >= static_cast<int>(ctx->cons.size())) return MCP_ERR_ARG;
  if (P) std::memcpy(P, ctx->cons[i].P, 12 * sizeof(double));
  if (Q) std::memcpy(Q, ctx->cons[i].Q, 12 * sizeof(double));
  if (target) std::memcpy(target, ctx->cons[i].target, 3 * sizeof(double));
  if (B) std::memcpy(B, ctx->cons[i].B, 12 * sizeof(double));
  return MCP_OK;
}

mcp_status mcp_load_obstacles(mcp_ctx *ctx, const double *spheres, int32_t n_spheres, const double *aabbs,
                              int32_t n_aabbs) {
  if (!ctx) return MCP_ERR_ARG;
  if (n_spheres < 0 || n_spheres > MCP_MAX_OBSTACLES || n_aabbs < 0 || n_aabbs > MCP_MAX_AABBS)
    return fail(ctx, MCP_ERR_ARG, "obstacle counts %d / %d outside [0, %d] / [0, %d]", n_spheres, n_aabbs,
                MCP_MAX_OBSTACLES, MCP_MAX_AABBS);
  if ((n_spheres && !spheres) || (n_aabbs && !aabbs)) return fail(ctx, MCP_ERR_ARG, "obstacle array is NULL");
  // non-finite values would make a chunk's bounding sphere hide its other
  // obstacles; rejected before anything is replaced
  for (int64_t i = 0; i < 4 * static_cast<int64_t>(n_spheres); ++i)
    if (!std::isfinite(spheres[i])) return fail(ctx, MCP_ERR_ARG, "obstacle sphere %lld is not finite", (long long)(i / 4));
  for (int64_t i = 0; i < 6 * static_cast<int64_t>(n_aabbs); ++i)
    if (!std::isfinite(aabbs[i])) return fail(ctx, MCP_ERR_ARG, "obstacle box %lld is not finite", (long long)(i / 6));
  DeviceGuard g(ctx->device);
  cudaFree(ctx->d_obs32);
  cudaFree(ctx->d_obs64);
  cudaFree(ctx->d_box32);
  cudaFree(ctx->d_box64);
  ctx->d_obs32 = nullptr;
  ctx->d_obs64 = nullptr;
  ctx->d_box32 = nullptr;
  ctx->d_box64 = nullptr;
  ctx->obs_loaded = false;
  const size_t n_o = static_cast<size_t>(n_spheres > 0 ? n_spheres : 1);
  const size_t n_b = static_cast<size_t>(n_aabbs > 0 ? n_aabbs : 1);
  // spatial order (Morton code of the centres), so that the chunks of
  // consecutive obstacles the check tests first are compact (scenes of more
  // than 32 obstacles; smaller ones keep the caller's order); the verdicts do
  // not depend on the order
  std::vector<double> sorted(spheres ? spheres : nullptr, spheres ? spheres + 4 * static_cast<size_t>(n_spheres) : nullptr);
  if (n_spheres > 32) {
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = spheres[a];
    for (int o = 1; o < n_spheres; ++o)
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], spheres[4 * o + a]);
        hi[a] = std::max(hi[a], spheres[4 * o + a]);
      }
    std::vector<std::pair<uint32_t, int>> key(static_cast<size_t>(n_spheres));
    for (int o = 0; o < n_spheres; ++o) {
      uint32_t code = 0;
      for (int a = 0; a < 3; ++a) {
        const double u = hi[a] > lo[a] ? (spheres[4 * o + a] - lo[a]) / (hi[a] - lo[a]) : 0.0;
        const uint32_t v = static_cast<uint32_t>(std::isfinite(u) ? std::min(std::max(u, 0.0), 1.0) * 1023.0 : 0.0);
        for (int b = 0; b < 10; ++b) code |= ((v >> b) & 1u) << (3 * b + a);
      }
      key[static_cast<size_t>(o)] = {code, o};
    }
    std::stable_sort(key.begin(), key.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
    for (int o = 0; o < n_spheres; ++o)
      for (int e = 0; e < 4; ++e) sorted[4 * static_cast<size_t>(o) + e] = spheres[4 * key[static_cast<size_t>(o)].second + e];
  }
  const size_t n_rec = n_o + static_cast<size_t>(obs_chunks(n_spheres));
  MCP_CUDA(dev_malloc(&ctx->d_obs32, n_rec * 2 * sizeof(float4), "obstacles"), "cudaMalloc obstacles");
  MCP_CUDA(dev_malloc(&ctx->d_obs64, n_o * 4 * sizeof(double), "obstacles"), "cudaMalloc obstacles");
  MCP_CUDA(dev_malloc(&ctx->d_box32, n_b * 6 * sizeof(float), "boxes"), "cudaMalloc boxes");
  MCP_CUDA(dev_malloc(&ctx->d_box64, n_b * 6 * sizeof(double), "boxes"), "cudaMalloc boxes");
  if (!ctx->d_origin) MCP_CUDA(dev_malloc(&ctx->d_origin, 3 * sizeof(double), "obstacle origin"), "cudaMalloc origin");
  if (n_spheres)
    MCP_CUDA(cudaMemcpy(ctx->d_obs64, sorted.data(), n_spheres * 4 * sizeof(double), cudaMemcpyHostToDevice), "copy");
  if (n_aabbs)
    MCP_CUDA(cudaMemcpy(ctx->d_box64, aabbs, n_aabbs * 6 * sizeof(double), cudaMemcpyHostToDevice), "copy");
  k_prep_obstacles<<<1, 256>>>(ctx->d_obs64, n_spheres, ctx->d_box64, n_aabbs, reinterpret_cast<float *>(ctx->d_obs32),
                               ctx->d_box32, ctx->d_origin);
  ctx->launches += 1;
  MCP_CUDA(cudaGetLastError(), "obstacle preparation launch");
  MCP_CUDA(cudaMemcpy(ctx->origin, ctx->d_origin, 3 * sizeof(double), cudaMemcpyDeviceToHost), "origin copy");
  ctx->hm.d_obs32 = ctx->d_obs32;
  ctx->hm.d_obs64 = ctx->d_obs64;
  ctx->hm.d_box32 = ctx->d_box32;
  ctx->hm.d_box64 = ctx->d_box64;
  ctx->hm.n_obs = n_spheres;
  ctx->hm.n_box = n_aabbs;
  ctx->obs_loaded = true;
  ++ctx->version;
  return update_shifted(ctx);
}

static mcp_status validate_params(mcp_ctx *ctx, const mcp_project_params *p) {
  if (!p) return fail(ctx, MCP_ERR_ARG, "params is NULL");
  if (!(p->tol > 0.0) || !std::isfinite(p->tol)) return fail(ctx, MCP_ERR_ARG, "tol must be positive");
  if (p->max_iters < 0 || p->max_iters > 255) return fail(ctx, MCP_ERR_ARG, "max_iters %d outside [0, 255]", p->max_iters);
  if (p->precision != 0 && p->precision != 1) return fail(ctx, MCP_ERR_ARG, "precision %d", p->precision);
  if (p->cyclic != 0 && p->cyclic != 1) return fail(ctx, MCP_ERR_ARG, "cyclic %d", p->cyclic);
  if (p->outer != 0 && p->outer != 1) return fail(ctx, MCP_ERR_ARG, "outer %d", p->outer);
  if (p->outer && p->cyclic) return fail(ctx, MCP_ERR_UNSUPPORTED, "the outer form takes stacked steps");
  if (!(p->alpha >= 0.0 && p->alpha <= 2.0)) return fail(ctx, MCP_ERR_ARG, "alpha must be in (0, 2] (0 = 1)");
  if (!(p->lambda >= 0.0) || !std::isfinite(p->lambda)) return fail(ctx, MCP_ERR_ARG, "lambda must be >= 0");
  if (!std::isfinite(p->max_step) || !std::isfinite(p->pivot_fp64)) return fail(ctx, MCP_ERR_ARG, "non-finite parameter");
  if (!ctx->robot_loaded || !ctx->cons_loaded) return fail(ctx, MCP_ERR_STATE, "robot and constraints must be loaded");
  if (ctx->prob_class < 0)
    return fail(ctx, MCP_ERR_UNSUPPORTED, "the loaded robot / constraint stack matches no compiled problem class");
  return MCP_OK;
}

static void fill_call(mcp_ctx *ctx, const mcp_project_params *p, ProjCall &c, cudaStream_t s) {
  c.precision = p->precision;
  c.tol = p->tol;
  c.cap = p->max_iters;
  c.lambda = p->lambda;
  c.max_step = p->max_step;
  c.pivot = p->pivot_fp64;
  c.cyclic = p->cyclic != 0;
  c.outer = p->outer != 0;
  c.alpha = p->alpha > 0.0 ? p->alpha : 1.0;
  c.counter = ctx->d_counter;
  c.tune = ctx->tune;
  c.stream = s;
}

mcp_status mcp_project_batch(mcp_ctx *ctx, const mcp_project_params *p, int64_t n, int64_t ld, const void *q_in,
                             void *q_out, uint8_t *flags, uint8_t *iters, double *resid, mcp_stream stream) {
  if (!ctx) return MCP_ERR_ARG;
  mcp_status st = validate_params(ctx, p);
  if (st != MCP_OK) return st;
  if (n < 0 || ld < n) return fail(ctx, MCP_ERR_ARG, "need 0 <= n <= ld (n = %lld, ld = %lld)", (long long)n, (long long)ld);
  if (n == 0) return MCP_OK;
  const char *names[5] = {"q_in", "q_out", "flags", "iters", "resid"};
  const void *ptrs[5] = {q_in, q_out, flags, iters, resid};
  for (int i = 0; i < 5; ++i)
    if ((st = check_batch_ptr(ctx, ptrs[i], names[i])) != MCP_OK) return st;
  DeviceGuard g(ctx->device);
  ProjCall c;
  fill_call(ctx, p, c, reinterpret_cast<cudaStream_t>(stream));
  c.q_in = q_in;
  c.ld_in = ld;
  c.total = n;
  c.q_out = q_out;
  c.ld_out = ld;
  c.flags = flags;
  c.iters = iters;
  c.resid = resid;
  int launches = 0;
  cudaError_t e = registry()[ctx->prob_class].project_fn(ctx->hm, c, &launches);
  ctx->launches += launches;
  if ((e = injected(ctx, e, "project_batch launch")) != cudaSuccess) return cuda_fail(ctx, e, "project_batch launch");
  return MCP_OK;
}

// Projection, then the check of its outputs: fused into the projection kernel
// when the autotuner found that faster for this problem, else a second launch.
static cudaError_t run_project_check(mcp_ctx *ctx, ProjCall c, int *launches) {
  const ClassDesc &cd = registry()[ctx->prob_class];
  c.fused_check = ctx->tune.fuse_check && !c.outer;
  if (c.fused_check) return cd.project_fn(ctx->hm, c, launches);
  cudaError_t e = cd.project_fn(ctx->hm, c, launches);
  if (e != cudaSuccess) return e;
  CheckCall k;
  k.precision = c.precision;
  k.n = c.total;
  k.ld = c.ld_out;
  k.q = c.q_out;
  k.out = c.hit;
  k.pairs = c.pairs;
  k.stream = c.stream;
  return cd.check_fn(ctx->hm, k, launches);
}

mcp_status mcp_project_check_batch(mcp_ctx *ctx, const mcp_project_params *p, int64_t n, int64_t ld,
                                   const void *q_in, void *q_out, uint8_t *flags, uint8_t *iters, double *resid,
                                   uint8_t *in_collision, uint32_t *pairs_tested, mcp_stream stream) {
  if (!ctx) return MCP_ERR_ARG;
  mcp_status st = validate_params(ctx, p);
  if (st != MCP_OK) return st;
  if (!ctx->obs_loaded) return fail(ctx, MCP_ERR_STATE, "obstacles must be loaded");
  if (n < 0 || ld < n) return fail(ctx, MCP_ERR_ARG, "need 0 <= n <= ld (n = %lld, ld = %lld)", (long long)n, (long long)ld);
  if (n == 0) return MCP_OK;
  const char *names[6] = {"q_in", "q_out", "flags", "iters", "resid", "in_collision"};
  const void *ptrs[6] = {q_in, q_out, flags, iters, resid, in_collision};
  for (int i = 0; i < 6; ++i)
    if ((st = check_batch_ptr(ctx, ptrs[i], names[i])) != MCP_OK) return st;
  if (pairs_tested && (st = check_batch_ptr(ctx, pairs_tested, "pairs_tested")) != MCP_OK) return st;
  DeviceGuard g(ctx->device);
  ProjCall c;
  fill_call(ctx, p, c, reinterpret_cast<cudaStream_t>(stream));
  c.q_in = q_in;
  c.ld_in = ld;
  c.total = n;
  c.q_out = q_out;
  c.ld_out = ld;
  c.flags = flags;
  c.iters = iters;
  c.resid = resid;
  c.hit = in_collision;
  c.pairs = pairs_tested;
  int launches = 0;
  cudaError_t e = run_project_check(ctx, c, &launches);
  ctx->launches += launches;
  if ((e = injected(ctx, e, "project_check_batch launch")) != cudaSuccess) return cuda_fail(ctx, e, "project_check_batch launch");
  return MCP_OK;
}

mcp_status mcp_extend_batch(mcp_ctx *ctx, const mcp_project_params *p, const mcp_extend_params *e, int64_t n_ext,
                            int64_t ld, const float *q_s, const float *q_t, const float *eps, int64_t ld_eps,
                            float *q_proj, uint8_t *status, int32_t *n_points, int32_t *winner, int32_t *steps,
                            mcp_stream stream) {
  if (!ctx) return MCP_ERR_ARG;
  mcp_status st = validate_params(ctx, p);
  if (st != MCP_OK) return st;
  if (!e) return fail(ctx, MCP_ERR_ARG, "extend params is NULL");
  if (p->precision != 0) return fail(ctx, MCP_ERR_ARG, "the extension runs the FP32 path (precision 0)");
  if (p->cyclic != 0 || p->outer != 0) return fail(ctx, MCP_ERR_ARG, "the extension uses the stacked inner step");
  if (!ctx->obs_loaded) return fail(ctx, MCP_ERR_STATE, "obstacles must be loaded");
  if (e->n < 1 || e->n > 32) return fail(ctx, MCP_ERR_ARG, "n = %d outside [1, 32]", e->n);
  if (!(e->r > 0.0) || !(e->delta > 0.0) || !std::isfinite(e->r) || !std::isfinite(e->delta))
    return fail(ctx, MCP_ERR_ARG, "r and delta must be positive");
  if (e->max_depth < 0 || e->max_depth > 16) return fail(ctx, MCP_ERR_ARG, "max_depth %d outside [0, 16]", e->max_depth);
  if (n_ext < 0 || ld < n_ext || ld_eps < n_ext) return fail(ctx, MCP_ERR_ARG, "need 0 <= n_ext <= ld, ld_eps");
  if (n_ext == 0) return MCP_OK;
  const char *names[7] = {"q_s", "q_t", "eps", "q_proj", "status", "n_points", "winner"};
  const void *ptrs[7] = {q_s, q_t, eps, q_proj, status, n_points, winner};
  for (int i = 0; i < 7; ++i)
    if ((st = check_batch_ptr(ctx, ptrs[i], names[i])) != MCP_OK) return st;
  if (steps && (st = check_batch_ptr(ctx, steps, "steps")) != MCP_OK) return st;
  DeviceGuard g(ctx->device);
  ExtCall c;
  c.tol = p->tol;
  c.cap = p->max_iters;
  c.lambda = p->lambda;
  c.max_step = p->max_step;
  c.pivot = p->pivot_fp64;
  c.alpha = p->alpha > 0.0 ? p->alpha : 1.0;
  c.r = e->r;
  c.delta = e->delta;
  c.n = e->n;
  c.max_depth = e->max_depth;
  c.n_ext = n_ext;
  c.ld = ld;
  c.ld_eps = ld_eps;
  c.q_s = q_s;
  c.q_t = q_t;
  c.eps = eps;
  c.q_proj = q_proj;
  c.status = status;
  c.n_points = n_points;
  c.winner = winner;
  c.steps = steps;
  c.counter = ctx->d_counter;
  c.scratch = &ctx->ext_scratch;
  c.stream = reinterpret_cast<cudaStream_t>(stream);
  int launches = 0;
  cudaError_t err = registry()[ctx->prob_class].extend_fn(ctx->hm, c, &launches);
  ctx->launches += launches;
  if ((err = injected(ctx, err, "extend_batch launch")) != cudaSuccess) return cuda_fail(ctx, err, "extend_batch launch");
  return MCP_OK;
}

mcp_status mcp_project_segments(mcp_ctx *ctx, const mcp_project_params *p, int64_t n_seg, int64_t ld_seg,
                                const void *start, const void *delta, const int32_t *len, int64_t total,
                                int64_t ld_out, void *q_out, uint8_t *flags, uint8_t *iters, double *resid,
                                mcp_stream stream) {
  if (!ctx) return MCP_ERR_ARG;
  mcp_status st = validate_params(ctx, p);
  if (st != MCP_OK) return st;
  if (n_seg < 0 || ld_seg < n_seg || n_seg > (1ll << 31) - 1)
    return fail(ctx, MCP_ERR_ARG, "need 0 <= n_seg <= ld_seg, n_seg < 2^31");
  if (total < 0 || ld_out < total) return fail(ctx, MCP_ERR_ARG, "need 0 <= total <= ld_out");
  if (n_seg == 0 || total == 0) return MCP_OK;
  const char *names[7] = {"start", "delta", "len", "q_out", "flags", "iters", "resid"};
  const void *ptrs[7] = {start, delta, len, q_out, flags, iters, resid};
  for (int i = 0; i < 7; ++i)
    if ((st = check_batch_ptr(ctx, ptrs[i], names[i])) != MCP_OK) return st;
  DeviceGuard g(ctx->device);
  if (ctx->seg_cap < n_seg + 1) {
    cudaFree(ctx->d_seg_off);
    ctx->d_seg_off = nullptr;
    ctx->seg_cap = 0;
    MCP_CUDA(dev_malloc(&ctx->d_seg_off, (n_seg + 1) * sizeof(long long), "segment offsets"), "cudaMalloc segment offsets");
    ctx->seg_cap = n_seg + 1;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  ProjCall c;
  fill_call(ctx, p, c, s);
  c.segments = true;
  c.start = start;
  c.delta = delta;
  c.ld_seg = ld_seg;
  c.seg_off = ctx->d_seg_off;
  c.n_seg = static_cast<int>(n_seg);
  c.total = total;
  c.q_out = q_out;
  c.ld_out = ld_out;
  c.flags = flags;
  c.iters = iters;
  c.resid = resid;
  const ClassDesc &cls = registry()[ctx->prob_class];
  // enqueue: scan of the lengths, counter reset + persistent kernel
  auto enqueue = [&](cudaStream_t st, int *launches) -> cudaError_t {
    k_scan_lengths<<<1, 1024, 0, st>>>(len, n_seg, ctx->d_seg_off);
    *launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ProjCall cc = c;
    cc.stream = st;
    return cls.project_fn(ctx->hm, cc, launches);
  };
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  MCP_CUDA(cudaStreamIsCapturing(s, &cs), "cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone) {  // the caller is capturing: enqueue directly into its graph
    int launches = 0;
    cudaError_t e = enqueue(s, &launches);
    ctx->launches += launches;
    if ((e = injected(ctx, e, "project_segments launch")) != cudaSuccess) return cuda_fail(ctx, e, "project_segments launch");
    return MCP_OK;
  }
  // key: everything the captured launches depend on
  std::vector<unsigned char> key;
  auto put = [&key](const void *v, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(v);
    key.insert(key.end(), b, b + n);
  };
  const void *key_ptrs[9] = {start, delta, len, q_out, flags, iters, resid, ctx->d_seg_off, ctx->d_counter};
  put(key_ptrs, sizeof(key_ptrs));
  const int64_t sizes[5] = {n_seg, ld_seg, total, ld_out, static_cast<int64_t>(ctx->version)};
  put(sizes, sizeof(sizes));
  put(p, sizeof(*p));
  put(&ctx->tune, sizeof(ctx->tune));
  if (!ctx->seg_exec || key != ctx->seg_key) {
    if (ctx->seg_exec) {
      cudaGraphExecDestroy(ctx->seg_exec);
      ctx->seg_exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    MCP_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    int launches = 0;
    cudaError_t e = enqueue(ctx->cap_stream, &launches);
    cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(ctx, e != cudaSuccess ? e : e2, "capture of the segment projection");
    }
    e = cudaGraphInstantiate(&ctx->seg_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      ctx->seg_exec = nullptr;
      return cuda_fail(ctx, e, "graph instantiation");
    }
    ctx->seg_key = std::move(key);
    ctx->seg_graph_launches = launches;
  }
  MCP_CUDA(cudaGraphLaunch(ctx->seg_exec, s), "graph launch");
  ctx->launches += ctx->seg_graph_launches;
  return MCP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free segment projection (mcp_project_segments_noalloc).
//
// The scratch of the segment projection -- the persistent kernel's work
// counter, then the exclusive prefix sums of the segment lengths -- lives in
// this file-scope device array instead of memory allocated per context.  Every
// GPU that loads the library holds it until the process exits; every call
// shares it.  In host code `g_noalloc_scratch` is only a stand-in for the
// symbol, not a device address: its address on each device is looked up once
// with cudaGetSymbolAddress, with that device current, and that pointer is
// what the kernels receive.
// ---------------------------------------------------------------------------
static __device__ __align__(256) long long g_noalloc_scratch[2 + MCP_NOALLOC_MAX_SEGMENTS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
long long *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).
cudaError_t noalloc_scratch(int device, long long **out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = static_cast<long long *>(p);
  }
  *out = g_noalloc_ptr[device];
  return cudaSuccess;
}
}  // namespace

extern "C" {

mcp_status mcp_project_segments_noalloc(mcp_ctx *ctx, const mcp_project_params *p, int64_t n_seg, int64_t ld_seg,
                                        const void *start, const void *delta, const int32_t *len, int64_t total,
                                        int64_t ld_out, void *q_out, uint8_t *flags, uint8_t *iters, double *resid,
                                        mcp_stream stream) {
  if (!ctx) return MCP_ERR_ARG;
  mcp_status st = validate_params(ctx, p);
  if (st != MCP_OK) return st;
  if (n_seg < 0 || ld_seg < n_seg) return fail(ctx, MCP_ERR_ARG, "need 0 <= n_seg <= ld_seg");
  if (n_seg > MCP_NOALLOC_MAX_SEGMENTS)
    return fail(ctx, MCP_ERR_ARG,
                "n_seg = %lld exceeds the allocation-free limit of %d segments; split the batch or use "
                "mcp_project_segments",
                (long long)n_seg, MCP_NOALLOC_MAX_SEGMENTS);
  if (total < 0 || ld_out < total) return fail(ctx, MCP_ERR_ARG, "need 0 <= total <= ld_out");
  if (n_seg == 0 || total == 0) return MCP_OK;
  const char *names[7] = {"start", "delta", "len", "q_out", "flags", "iters", "resid"};
  const void *ptrs[7] = {start, delta, len, q_out, flags, iters, resid};
  for (int i = 0; i < 7; ++i)
    if ((st = check_batch_ptr(ctx, ptrs[i], names[i])) != MCP_OK) return st;
  DeviceGuard g(ctx->device);
  long long *scratch = nullptr;
  MCP_CUDA(noalloc_scratch(ctx->device, &scratch), "cudaGetSymbolAddress of the allocation-free scratch");
  unsigned long long *counter = reinterpret_cast<unsigned long long *>(scratch);
  long long *offsets = scratch + 1;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_scan_lengths<<<1, 1024, 0, s>>>(len, n_seg, offsets);  // writes offsets[0 .. n_seg]
  ctx->launches += 1;
  MCP_CUDA(cudaGetLastError(), "segment scan launch");
  ProjCall c;
  fill_call(ctx, p, c, s);
  c.counter = counter;  // cleared on the stream by the projection launcher before its kernel
  c.segments = true;
  c.start = start;
  c.delta = delta;
  c.ld_seg = ld_seg;
  c.seg_off = offsets;
  c.n_seg = static_cast<int>(n_seg);
  c.total = total;
  c.q_out = q_out;
  c.ld_out = ld_out;
  c.flags = flags;
  c.iters = iters;
  c.resid = resid;
  int launches = 0;
  cudaError_t e = registry()[ctx->prob_class].project_fn(ctx->hm, c, &launches);
  ctx->launches += launches;
  if ((e = injected(ctx, e, "project_segments_noalloc launch")) != cudaSuccess) return cuda_fail(ctx, e, "project_segments_noalloc launch");
  return MCP_OK;
}

mcp_status mcp_check_batch(mcp_ctx *ctx, int64_t n, int64_t ld, const void *q, int32_t precision,
                           uint8_t *in_collision, uint32_t *pairs_tested, mcp_stream stream) {
  if (!ctx) return MCP_ERR_ARG;
  if (!ctx->robot_loaded) return fail(ctx, MCP_ERR_STATE, "robot not loaded");
  if (!ctx->obs_loaded) return fail(ctx, MCP_ERR_STATE, "obstacles not loaded");
  if (ctx->robot_class < 0) return fail(ctx, MCP_ERR_UNSUPPORTED, "the loaded robot matches no compiled problem class");
  if (precision != 0 && precision != 1) return fail(ctx, MCP_ERR_ARG, "precision %d", precision);
  if (n < 0 || ld < n) return fail(ctx, MCP_ERR_ARG, "need 0 <= n <= ld");
  if (n == 0) return MCP_OK;
  mcp_status st;
  if ((st = check_batch_ptr(ctx, q, "q")) != MCP_OK) return st;
  if ((st = check_batch_ptr(ctx, in_collision, "in_collision")) != MCP_OK) return st;
  if (pairs_tested && (st = check_batch_ptr(ctx, pairs_tested, "pairs_tested")) != MCP_OK) return st;
  DeviceGuard g(ctx->device);
  CheckCall c;
  c.pairs = pairs_tested;
  c.precision = precision;
  c.n = n;
  c.ld = ld;
  c.q = q;
  c.out = in_collision;
  c.stream = reinterpret_cast<cudaStream_t>(stream);
  int launches = 0;
  cudaError_t e = registry()[ctx->robot_class].check_fn(ctx->hm, c, &launches);
  ctx->launches += launches;
  if ((e = injected(ctx, e, "check_batch launch")) != cudaSuccess) return cuda_fail(ctx, e, "check_batch launch");
  return MCP_OK;
}

mcp_status mcp_project_vjp(mcp_ctx *ctx, int64_t n, int64_t ld, const float *q_star, const float *g, float *out,
                           uint8_t *flags, mcp_stream stream) {
  if (!ctx) return MCP_ERR_ARG;
  if (!ctx->robot_loaded || !ctx->cons_loaded) return fail(ctx, MCP_ERR_STATE, "robot and constraints must be loaded");
  if (ctx->prob_class < 0) return fail(ctx, MCP_ERR_UNSUPPORTED, "no compiled problem class for this stack");
  if (n < 0 || ld < n) return fail(ctx, MCP_ERR_ARG, "need 0 <= n <= ld");
  if (n == 0) return MCP_OK;
  mcp_status st;
  if ((st = check_batch_ptr(ctx, q_star, "q_star")) != MCP_OK) return st;
  if ((st = check_batch_ptr(ctx, g, "g")) != MCP_OK) return st;
  if ((st = check_batch_ptr(ctx, out, "out")) != MCP_OK) return st;
  if (flags && (st = check_batch_ptr(ctx, flags, "flags")) != MCP_OK) return st;
  DeviceGuard gd(ctx->device);
  VjpCall c;
  c.n = n;
  c.ld = ld;
  c.q = q_star;
  c.g = g;
  c.out = out;
  c.flags = flags;
  c.stream = reinterpret_cast<cudaStream_t>(stream);
  int launches = 0;
  cudaError_t e = registry()[ctx->prob_class].vjp_fn(ctx->hm, c, &launches);
  ctx->launches += launches;
  if ((e = injected(ctx, e, "project_vjp launch")) != cudaSuccess) return cuda_fail(ctx, e, "project_vjp launch");
  return MCP_OK;
}

mcp_status mcp_path_length_grad(mcp_ctx *ctx, int64_t n_paths, int32_t n_way, int64_t ld, const float *Q,
                                float *length, float *grad, mcp_stream stream) {
  if (!ctx) return MCP_ERR_ARG;
  if (!ctx->robot_loaded) return fail(ctx, MCP_ERR_STATE, "robot not loaded");
  if (n_paths < 0 || n_way < 1 || ld < n_paths * n_way) return fail(ctx, MCP_ERR_ARG, "need ld >= n_paths * n_way");
  if (n_paths == 0) return MCP_OK;
  mcp_status st;
  if ((st = check_batch_ptr(ctx, Q, "Q")) != MCP_OK) return st;
  if (length && (st = check_batch_ptr(ctx, length, "length")) != MCP_OK) return st;
  if (grad && (st = check_batch_ptr(ctx, grad, "grad")) != MCP_OK) return st;
  DeviceGuard gd(ctx->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int d = ctx->robot.nj;
  if (grad) {
    const long long n = n_paths * n_way;
    k_path_grad<<<static_cast<unsigned>((n + 127) / 128), 128, 0, s>>>(Q, ld, n_paths, n_way, d, grad);
    ctx->launches += 1;
    MCP_CUDA(cudaGetLastError(), "path gradient launch");
  }
  if (length) {
    k_path_length<<<static_cast<unsigned>((n_paths * 32 + 127) / 128), 128, 0, s>>>(Q, ld, n_paths, n_way, d, length);
    ctx->launches += 1;
    MCP_CUDA(cudaGetLastError(), "path length launch");
  }
  return MCP_OK;
}

mcp_status mcp_fma_probe(mcp_ctx *ctx, int32_t precision, int64_t iters, void *out, int64_t *flops,
                         mcp_stream stream) {
  if (!ctx) return MCP_ERR_ARG;
  if (precision != 0 && precision != 1) return fail(ctx, MCP_ERR_ARG, "precision must be 0 (FP32) or 1 (FP64)");
  if (iters < 1 || iters > (int64_t(1) << 32)) return fail(ctx, MCP_ERR_ARG, "iters outside [1, 2^32]");
  if (!out) return fail(ctx, MCP_ERR_ARG, "out is NULL");
  mcp_status st;
  if ((st = check_batch_ptr(ctx, out, "out")) != MCP_OK) return st;
  DeviceGuard gd(ctx->device);
  int sms = 0;
  MCP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "device attribute");
  const unsigned blocks = static_cast<unsigned>(sms) * 8u;  // 2048 threads per SM
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (precision == 0)
    k_fma_probe<float><<<blocks, 256, 0, s>>>(static_cast<float *>(out), iters, 0.999f, 1e-3f);
  else
    k_fma_probe<double><<<blocks, 256, 0, s>>>(static_cast<double *>(out), iters, 0.999, 1e-3);
  ctx->launches += 1;
  MCP_CUDA(cudaGetLastError(), "fma probe launch");
  if (flops) *flops = static_cast<int64_t>(blocks) * 256 * 8 * 2 * iters;
  return MCP_OK;
}

mcp_status mcp_path_step(mcp_ctx *ctx, int64_t n_paths, int32_t n_way, int64_t ld, float *Q, const float *D, float eta,
                         float max_step, mcp_stream stream) {
  if (!ctx) return MCP_ERR_ARG;
  if (!ctx->robot_loaded) return fail(ctx, MCP_ERR_STATE, "robot not loaded");
  if (n_paths < 0 || n_way < 1 || ld < n_paths * n_way) return fail(ctx, MCP_ERR_ARG, "need ld >= n_paths * n_way");
  if (!std::isfinite(eta) || !std::isfinite(max_step)) return fail(ctx, MCP_ERR_ARG, "non-finite step parameters");
  if (n_paths == 0) return MCP_OK;
  mcp_status st;
  if ((st = check_batch_ptr(ctx, Q, "Q")) != MCP_OK) return st;
  if ((st = check_batch_ptr(ctx, D, "D")) != MCP_OK) return st;
  DeviceGuard gd(ctx->device);
  const long long n = n_paths * n_way;
  k_path_step<<<static_cast<unsigned>((n + 127) / 128), 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      Q, D, ld, n_paths, n_way, ctx->robot.nj, eta, max_step);
  ctx->launches += 1;
  MCP_CUDA(cudaGetLastError(), "path step launch");
  return MCP_OK;
}

mcp_status mcp_set_tuning(mcp_ctx *ctx, int32_t tpb, int32_t blocks_per_sm, int32_t chunk, int32_t fuse_check,
                          int32_t threads_per_config) {
  if (!ctx) return MCP_ERR_ARG;
  if ((tpb != 64 && tpb != 128 && tpb != 256) || blocks_per_sm < 1 || blocks_per_sm > 8 ||
      tpb * blocks_per_sm > 2048 || chunk < 1 || chunk > 64 || (fuse_check != 0 && fuse_check != 1) ||
      (threads_per_config != 1 && threads_per_config != 2))
    return fail(ctx, MCP_ERR_ARG, "tuning (%d, %d, %d, %d, %d) outside the supported shapes", tpb, blocks_per_sm, chunk,
                fuse_check, threads_per_config);
  ctx->tune = Tuning{tpb, blocks_per_sm, chunk, fuse_check == 1, threads_per_config};
  ctx->tuned = true;
  return MCP_OK;
}

mcp_status mcp_autotune(mcp_ctx *ctx, const mcp_project_params *p, int64_t n_sample, int64_t ld, const void *q_sample,
                        int32_t *tpb_out, int32_t *bps_out, int32_t *chunk_out, int32_t *fuse_out,
                        int32_t *tpc_out, mcp_stream stream) {
  if (!ctx) return MCP_ERR_ARG;
  mcp_status st = validate_params(ctx, p);
  if (st != MCP_OK) return st;
  if (p->precision != 0) return fail(ctx, MCP_ERR_ARG, "autotune applies to the FP32 projection (precision 0)");
  if (n_sample < 1 || ld < n_sample) return fail(ctx, MCP_ERR_ARG, "need 1 <= n_sample <= ld");
  if ((st = check_batch_ptr(ctx, q_sample, "q_sample")) != MCP_OK) return st;
  DeviceGuard g(ctx->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int d = ctx->robot.nj;
  float *out = nullptr;
  uint8_t *fl = nullptr, *it = nullptr, *hit = nullptr;
  double *res = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = dev_malloc(&out, sizeof(float) * d * ld, "autotune buffers");
  if (err == cudaSuccess) err = dev_malloc(&fl, ld, "autotune buffers");
  if (err == cudaSuccess) err = dev_malloc(&hit, ld, "autotune buffers");
  if (err == cudaSuccess) err = dev_malloc(&it, ld, "autotune buffers");
  if (err == cudaSuccess) err = dev_malloc(&res, sizeof(double) * ld, "autotune buffers");
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  const Tuning saved = ctx->tune;
  Tuning best = saved;
  float best_ms = 1e30f;
  const int tpbs[3] = {64, 128, 256};
  const int bpss[4] = {1, 2, 4, 8};
  const int chunks[3] = {16, 32, 64};
  // With obstacles loaded the step that matters is projection + check: every
  // launch shape is timed both fused and as two launches.  Each candidate's
  // time is the median of five bursts of four back-to-back calls (one
  // warm-up burst first): single calls sit near the resolution of the events.
  const int n_fuse = ctx->obs_loaded ? 2 : 1;
  // threads per configuration: 1, and 2 where the class has a pair kernel
  const int n_tpc = registry()[ctx->prob_class].pair ? 2 : 1;
  auto time_candidate = [&](float &med) -> cudaError_t {
    constexpr int BURSTS = 6, CALLS = 4;
    float times[BURSTS - 1];
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < BURSTS && e == cudaSuccess; ++r) {
      e = cudaEventRecord(e0, s);
      for (int k = 0; k < CALLS && e == cudaSuccess; ++k) {
        ProjCall call;
        fill_call(ctx, p, call, s);
        call.q_in = q_sample;
        call.ld_in = ld;
        call.total = n_sample;
        call.q_out = out;
        call.ld_out = ld;
        call.flags = fl;
        call.iters = it;
        call.resid = res;
        int launches = 0;
        if (ctx->obs_loaded) {
          call.hit = hit;
          e = run_project_check(ctx, call, &launches);
        } else {
          e = registry()[ctx->prob_class].project_fn(ctx->hm, call, &launches);
        }
        ctx->launches += launches;
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) times[r - 1] = ms;
    }
    if (e == cudaSuccess) {
      std::sort(times, times + (BURSTS - 1));
      med = times[(BURSTS - 1) / 2];
    }
    return e;
  };
  for (int a = 0; a < 3 && err == cudaSuccess; ++a)
    for (int b = 0; b < 4 && err == cudaSuccess; ++b)
      for (int c = 0; c < 3 && err == cudaSuccess; ++c)
        for (int f = 0; f < n_fuse && err == cudaSuccess; ++f)
          for (int t = 1; t <= n_tpc && err == cudaSuccess; ++t) {
            if (tpbs[a] * bpss[b] > 2048) continue;
            ctx->tune = Tuning{tpbs[a], bpss[b], chunks[c], f == 1, t};
            float med = 0.f;
            err = time_candidate(med);
            if (err == cudaSuccess && med < best_ms) {
              best_ms = med;
              best = ctx->tune;
            }
          }
  cudaFree(out);
  cudaFree(fl);
  cudaFree(it);
  cudaFree(hit);
  cudaFree(res);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    ctx->tune = saved;
    return cuda_fail(ctx, err, "autotune");
  }
  ctx->tune = best;
  ctx->tuned = true;
  if (tpb_out) *tpb_out = best.tpb;
  if (bps_out) *bps_out = best.blocks_per_sm;
  if (chunk_out) *chunk_out = best.chunk;
  if (fuse_out) *fuse_out = best.fuse_check ? 1 : 0;
  if (tpc_out) *tpc_out = best.tpc;
  return MCP_OK;
}

}  // extern "C"
