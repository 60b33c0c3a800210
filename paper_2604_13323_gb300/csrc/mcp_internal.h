// Host-side structures shared by the C ABI (mcp_api.cu) and the per-class
// kernel instantiations (inst_*.cu).  Not part of the public interface.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "mcp_device.cuh"

namespace mcp {

// Every device allocation of the library goes through this function: it
// counts them (mcp_alloc_count) and, for host-side failure tests, fails with
// cudaErrorMemoryAllocation every allocation whose label contains the text of
// the environment variable MCP_TEST_FAIL_ALLOC (unset or empty: never).
cudaError_t dev_malloc(void **p, size_t bytes, const char *label);
template <typename T>
cudaError_t dev_malloc(T **p, size_t bytes, const char *label) {
  return dev_malloc(reinterpret_cast<void **>(p), bytes, label);
}

// Bounds-check mode: the per-module error readers (see mcp_device.cuh).
void register_bounds_reader(unsigned int (*reader)(bool));
unsigned int bounds_error_of_all_modules(bool reset);

constexpr int MAXS = 256;  // robot spheres per robot

// Robot spheres sorted by the joint they ride on: spheres of link l (l = -1
// for world-fixed ones) are s[off[l + 1]] .. s[off[l + 2] - 1].
template <typename T>
struct SphereTable {
  T s[MAXS][4];
  T lb[MAXJ + 1][4];    // per link (index MAXJ: world-fixed spheres): bounding sphere, local centre + radius
  int16_t off[MAXJ + 2];
};

struct Tuning {
  int tpb = 128;          // threads per block of the persistent kernel
  int blocks_per_sm = 4;  // resident blocks per SM
  int chunk = 32;         // configurations a warp claims per atomic
  bool fuse_check = false;  // project_check_batch: check inside the projection kernel (else a second launch)
  int tpc = 1;              // threads per configuration: 2 = one lane per chain (classes with a pair kernel)
};

// What the collision check of the fused projection kernel reads from device
// memory: the model in the collision frame and the robot's spheres.
struct CheckData {
  ModelT<float> m;
  SphereTable<float> st;
};

struct HostModel {
  ModelT<float> m32;
  ModelT<float> m32_shifted;  // m32 in the collision frame (origin at the obstacle centroid)
  ModelT<double> m64;
  SphereTable<float> st32;
  SphereTable<double> st64;
  const ModelT<double> *d_m64 = nullptr;  // device copy of m64
  const double2 *d_tab = nullptr;         // FP64 sin/cos tables: 256 + 4097 entries
  const float4 *d_obs32 = nullptr;        // per obstacle 2 x float4: (-2c, |c|^2 - r^2), (-2r, 0, 0, 0), shifted
  const double *d_obs64 = nullptr;        // [n_obs * 4]
  const float *d_box32 = nullptr;         // [n_box * 6] lo.xyz, hi.xyz, shifted
  const double *d_box64 = nullptr;        // [n_box * 6]
  const CheckData *d_chk = nullptr;       // device copy of (m32_shifted, st32)
  int n_obs = 0;
  int n_box = 0;
  int sm_count = 1;
};

struct ProjCall {
  int precision = 0;
  double tol = 1e-5;
  int cap = 30;
  double lambda = 0.0;
  double max_step = 0.0;
  double pivot = 1e-7;
  bool cyclic = false;  // cyclic getDescentStep (one step per constraint per sweep)
  bool outer = false;   // outer form (J^T J + lambda I)^-1 J^T F
  double alpha = 1.0;   // step scale
  bool segments = false;
  // batch source
  const void *q_in = nullptr;
  long long ld_in = 0;
  // segment source
  const void *start = nullptr;
  const void *delta = nullptr;
  long long ld_seg = 0;
  const long long *seg_off = nullptr;  // [n_seg + 1] exclusive prefix sums (device)
  int n_seg = 0;
  long long total = 0;
  // outputs
  void *q_out = nullptr;
  long long ld_out = 0;
  uint8_t *flags = nullptr;
  uint8_t *iters = nullptr;
  double *resid = nullptr;
  // fused collision check of every output (project_check_batch)
  bool fused_check = false;
  uint8_t *hit = nullptr;
  uint32_t *pairs = nullptr;
  unsigned long long *counter = nullptr;  // zeroed work counter (device)
  Tuning tune;
  cudaStream_t stream = 0;
};

struct CheckCall {
  int precision = 0;
  long long n = 0, ld = 0;
  const void *q = nullptr;
  uint8_t *out = nullptr;
  uint32_t *pairs = nullptr;
  cudaStream_t stream = 0;
};

struct VjpCall {
  long long n = 0, ld = 0;
  const float *q = nullptr;
  const float *g = nullptr;
  float *out = nullptr;
  uint8_t *flags = nullptr;
  double pivot = 1e-7;
  cudaStream_t stream = 0;
};

// Device scratch owned by a context and grown by the launcher that needs it.
struct ScratchBuf {
  float *ptr = nullptr;
  size_t floats = 0;
};

struct ExtCall {
  double tol = 1e-5;
  int cap = 30;
  double lambda = 0.0;
  double max_step = 0.0;
  double pivot = 1e-7;
  double alpha = 1.0;
  double r = 0.3, delta = 0.02;
  int n = 8, max_depth = 6;
  long long n_ext = 0, ld = 0, ld_eps = 0;
  const float *q_s = nullptr;
  const float *q_t = nullptr;
  const float *eps = nullptr;
  float *q_proj = nullptr;
  uint8_t *status = nullptr;
  int32_t *n_points = nullptr;
  int32_t *winner = nullptr;
  int32_t *steps = nullptr;
  unsigned long long *counter = nullptr;
  ScratchBuf *scratch = nullptr;  // validated chains, one pair per resident group of lanes
  cudaStream_t stream = 0;
};

// Launchers, one explicit instantiation per problem class.  Each returns the
// CUDA error of its launch and adds the number of kernels it launched.
template <class P>
cudaError_t launch_project(const HostModel &hm, const ProjCall &c, int *launches);
template <class P>
cudaError_t launch_check(const HostModel &hm, const CheckCall &c, int *launches);
template <class P>
cudaError_t launch_vjp(const HostModel &hm, const VjpCall &c, int *launches);
template <class P>
cudaError_t launch_extend(const HostModel &hm, const ExtCall &c, int *launches);

}  // namespace mcp
