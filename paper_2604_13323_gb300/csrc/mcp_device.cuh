// Device building blocks of the projection path: model layout, sin/cos,
// 3x4 pose algebra, forward kinematics specialised on a compile-time robot
// structure, the SO(3) log map, and a fixed-size Cholesky solve.
//
// The paper traces robot kinematics and constraint functions into branch-free,
// loop-unrolled straight-line code for a robot known a priori (Sec. IV-A,
// "Tracing Compiler for Constraints"; Sec. VI).  Here the same effect comes
// from C++ templates: a problem class fixes the tree topology, the joint types,
// the structural zeros of each fixed joint offset (signed-permutation
// rotations, sparse translations) and the stacked constraint kinds at compile
// time, while every numeric value stays runtime data.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

#include <cuda_runtime.h>

namespace mcp {

// ---------------------------------------------------------------------------
// Bounds-check mode (debug builds compiled with -DMCP_CHECK_BOUNDS): the
// persistent kernels test the index of every batch-array access against the
// array's extent; an access out of range is skipped (loads read 0) and the
// source line of the first one is recorded in this module's error word,
// which mcp_bounds_status() reads.  Nothing traps.  In normal builds the test
// is the constant true and costs nothing.
// ---------------------------------------------------------------------------
#ifdef MCP_CHECK_BOUNDS
static __device__ unsigned int g_bounds_error;
__device__ __forceinline__ bool in_bounds(long long i, long long n, int line) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&g_bounds_error, 0u, static_cast<unsigned int>(line));
  return false;
}
#define MCP_CHK(i, n) ::mcp::in_bounds((i), (n), __LINE__)
// each module registers a reader of its own error word with the library
unsigned int bounds_error_of_all_modules(bool reset);
void register_bounds_reader(unsigned int (*reader)(bool));
static unsigned int read_bounds_error(bool reset) {
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_bounds_error, sizeof(v)) != cudaSuccess) v = ~0u;
  if (reset) {
    const unsigned int z = 0;
    cudaMemcpyToSymbol(g_bounds_error, &z, sizeof(z));
  }
  return v;
}
struct BoundsRegistration {
  BoundsRegistration() { register_bounds_reader(&read_bounds_error); }
};
static BoundsRegistration g_bounds_registration;
#else
#define MCP_CHK(i, n) true
#endif

constexpr int MAXJ = 40;
constexpr int MAXF = 8;
constexpr int MAXC = 8;
constexpr int MAXK = 24;
// The collision check's broad phase first tests a bounding sphere of each
// chunk of OBS_CHUNK consecutive obstacles (stored in spatial order).
constexpr int OBS_CHUNK = 16;
__host__ __device__ constexpr int obs_chunks(int n_obs) { return (n_obs + OBS_CHUNK - 1) / OBS_CHUNK; }

enum : int { REV = 0, PRIS = 1 };
enum : int {
  K_SPHERE = 0, K_AXIS = 1, K_POSE = 2, K_REL = 3, K_COM = 4,
  K_PLANE = 5,  // origin of frame a on the xy-plane of the task frame P
  K_LINE = 6,   // origin of frame a on the z-axis of the task frame P
  K_DIST = 7,   // |x_b - x_a| = L (closed linkage)
  K_PBND = 8,   // bounded TSR: Eq. 1 error outside the bounds B^w
  K_HULL = 9    // CoM xy distance to the support polygon (zero inside)
};
enum : uint32_t {
  FL_CONV = 1, FL_CAP = 2, FL_DIV = 4, FL_NONFINITE = 8, FL_RESOLVE = 16, FL_ACCEPT_FAIL = 32, FL_LIMITS = 64
};

// Model data in one precision.  3x4 transforms are row-major (column 3 = translation).
template <typename T>
struct ModelT {
  T X[MAXJ][12];      // fixed parent -> joint offsets
  T fX[MAXF][12];     // task-frame offsets
  T mass[MAXJ];
  T com[MAXJ][3];
  T lower[MAXJ];
  T upper[MAXJ];
  T cPinv[MAXC][12];  // POSE: (T_w^0)^-1; REL_POSE: T_ref^-1
  T cQinv[MAXC][12];  // POSE: (T_e^w)^-1
  T ctgt[MAXC][4];    // SPHERE radius; COM target xy; DIST length
  T cB[MAXC][12];     // PBND: lower[6], upper[6] of [t; log R]; HULL: polygon x0 y0 x1 y1 ... (CCW)
  T msub[MAXJ];       // mass of the subtree below (and including) joint j
  T inv_mass;         // 1 / total mass
  T shift[3];         // collision frame: world coordinates minus this origin (root offsets are pre-shifted)
};

// ---------------------------------------------------------------------------
// compile-time loop
// ---------------------------------------------------------------------------
template <class F, int... Is>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F &&f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------------------
// sin / cos
// ---------------------------------------------------------------------------
// FP32: Cody-Waite reduction by pi/2 (three-part split of pi/2) and Taylor
// polynomials of sin and cos on |r| <= pi/4, truncated where the next term is
// below 1e-9.  Accurate to a few ulp for the joint-angle range (|x| < 1e4).
__device__ __forceinline__ void sincos_f32(float x, float &s, float &c) {
  const float two_over_pi = 0.636619772367581343f;
  float k = rintf(x * two_over_pi);
  // pi/2 = 1.5703125 + 4.837512969970703e-4 + 7.549790126404332e-8 (+ 1.7e-15);
  // the first two parts have 12 significant bits, so k * part is exact.
  float r = fmaf(-k, 1.5703125f, x);
  r = fmaf(-k, 4.837512969970703e-4f, r);
  r = fmaf(-k, 7.549790126404332e-8f, r);
  float r2 = r * r;
  // sin r = r + r^3 (-1/3! + r^2 (1/5! + r^2 (-1/7! + r^2 / 9!)))
  float ps = fmaf(r2, 2.75573192e-6f, -1.98412698e-4f);
  ps = fmaf(r2, ps, 8.33333333e-3f);
  ps = fmaf(r2, ps, -1.66666667e-1f);
  float sr = fmaf(r * r2, ps, r);
  // cos r = 1 + r^2 (-1/2 + r^2 (1/4! + r^2 (-1/6! + r^2 (1/8! - r^2 / 10!))))
  float pc = fmaf(r2, -2.75573192e-7f, 2.48015873e-5f);
  pc = fmaf(r2, pc, -1.38888889e-3f);
  pc = fmaf(r2, pc, 4.16666667e-2f);
  pc = fmaf(r2, pc, -0.5f);
  float cr = fmaf(r2, pc, 1.0f);
  int qd = static_cast<int>(k) & 3;
  float ss = (qd & 1) ? cr : sr;
  float cc = (qd & 1) ? sr : cr;
  s = (qd & 2) ? -ss : ss;
  c = ((qd + 1) & 2) ? -cc : cc;
}

// FP64, table-driven argument reduction (Tang's method): x = k * 2pi/256 + r,
// |r| <= pi/256 (+ slack), sin/cos(k * 2pi/256) from a 256-entry table built
// once per context with sincospi, and Taylor polynomials of sin r (to r^7) and
// cos r (to r^6), whose next terms are below 1e-19.  k is chosen in FP32 (it
// only has to be close to the nearest integer), so the FP64 pipe sees 13 ops.
// The table index is masked, so any input stays in bounds.
__device__ __forceinline__ void sincos_f64_table(double x, const double2 *__restrict__ tab, double &s, double &c) {
  const float inv_step = 40.7436654315252059f;  // 256 / (2 pi)
  float kf = rintf(static_cast<float>(x) * inv_step);
  double k = static_cast<double>(kf);
  // 2 pi / 256 = head (32 significant bits, so k * head is exact) + tail (+ 5.5e-29)
  double r = fma(-k, 0.024543692605220713, x);
  r = fma(-k, 9.495469541415925e-13, r);
  double r2 = r * r;
  double ps = fma(r2, -1.9841269841269841e-04, 8.3333333333333333e-03);
  ps = fma(r2, ps, -1.6666666666666667e-01);
  double sr = fma(r * r2, ps, r);
  double pc = fma(r2, -1.3888888888888889e-03, 4.1666666666666667e-02);
  pc = fma(r2, pc, -0.5);
  double cr = fma(r2, pc, 1.0);
  double2 t = __ldg(&tab[static_cast<int>(kf) & 255]);  // (sin, cos) of k * 2pi/256
  s = fma(t.x, cr, t.y * sr);
  c = fma(t.y, cr, -(t.x * sr));
}

// FP64 sin/cos of an argument that is exactly an FP32 value (the acceptance
// pass evaluates F at the FP32 iterate).  x = h + r with h = m / 512 (m an
// integer, |m| <= 2048) and r = x - h, exact in FP32 (|r| <= 2^-10, and r is
// a multiple of x's ulp); sin and cos of h come from a table built once per
// context with CUDA's sincos, those of r from
//   sin r = r - r^3 / 6          (first omitted term r^5/120 <= 7.6e-18),
//   cos r - 1 = -r^2/2 + r^4/24  (first omitted term r^6/720 <= 1.3e-21),
// and the angle-addition formulas combine them: 10 FP64 operations and no
// argument reduction.  The truncation error stays below 2^-56 in absolute
// terms, under the rounding of the residual's O(1) intermediate values.
// Arguments outside [-4, 4] (or not finite) take the table-driven path above.
constexpr int SPLIT_TAB_OFF = 256;   // entries [256, 256 + 4097): (sin, cos)(m / 512), m = -2048..2048
constexpr int SPLIT_TAB_HALF = 2048;
__device__ __forceinline__ void sincos_f64_split_f(float xf, const double2 *__restrict__ tab, double &s, double &c) {
  const float mf = rintf(xf * 512.0f);
  if (fabsf(mf) <= static_cast<float>(SPLIT_TAB_HALF)) {
    const double r = static_cast<double>(fmaf(-mf, 0.001953125f, xf));  // exact
    const double2 t = __ldg(&tab[SPLIT_TAB_OFF + SPLIT_TAB_HALF + static_cast<int>(mf)]);
    const double r2 = r * r;
    const double sr = fma(r * r2, -1.6666666666666667e-01, r);
    const double cm = r2 * fma(r2, 4.1666666666666667e-02, -0.5);
    s = fma(t.x, cm, fma(t.y, sr, t.x));
    c = fma(t.y, cm, fma(-t.x, sr, t.y));
  } else {
    sincos_f64_table(static_cast<double>(xf), tab, s, c);
  }
}
__device__ __forceinline__ void sincos_f64_split(double x, const double2 *__restrict__ tab, double &s, double &c) {
  sincos_f64_split_f(static_cast<float>(x), tab, s, c);  // x holds an FP32 value
}

// Precision policies: the scalar type and the sin/cos routine.
struct OpsF32 {
  using T = float;
  const double2 *tab;
  __device__ __forceinline__ void sincos(float x, float &s, float &c) const { sincos_f32(x, s, c); }
  __device__ __forceinline__ static float sqrt_(float v) { return sqrtf(v); }
  __device__ __forceinline__ static float rsqrt_(float v) { return rsqrtf(v); }
  __device__ __forceinline__ static float atan2_(float y, float x) { return atan2f(y, x); }
};
struct OpsF64Table {  // FP64 acceptance / re-solve inside the FP32 path
  using T = double;
  const double2 *tab;
  __device__ __forceinline__ void sincos(double x, double &s, double &c) const { sincos_f64_table(x, tab, s, c); }
  __device__ __forceinline__ static double sqrt_(double v) { return sqrt(v); }
  __device__ __forceinline__ static double rsqrt_(double v) { return 1.0 / sqrt(v); }
  __device__ __forceinline__ static double atan2_(double y, double x) { return atan2(y, x); }
};
struct OpsF64Split {  // FP64 residual of an FP32 iterate (acceptance): arguments are FP32 values
  using T = double;
  const double2 *tab;
  __device__ __forceinline__ void sincos(double x, double &s, double &c) const { sincos_f64_split(x, tab, s, c); }
  __device__ __forceinline__ void sincos(float x, double &s, double &c) const { sincos_f64_split_f(x, tab, s, c); }
  __device__ __forceinline__ static double sqrt_(double v) { return sqrt(v); }
  __device__ __forceinline__ static double rsqrt_(double v) { return 1.0 / sqrt(v); }
  __device__ __forceinline__ static double atan2_(double y, double x) { return atan2(y, x); }
};
struct OpsF64Plain {  // the plain FP64 kernel: CUDA's double-precision math throughout
  using T = double;
  const double2 *tab;
  __device__ __forceinline__ void sincos(double x, double &s, double &c) const { ::sincos(x, &s, &c); }
  __device__ __forceinline__ static double sqrt_(double v) { return sqrt(v); }
  __device__ __forceinline__ static double rsqrt_(double v) { return 1.0 / sqrt(v); }
  __device__ __forceinline__ static double atan2_(double y, double x) { return atan2(y, x); }
};

template <typename T>
__device__ __forceinline__ T fma_(T a, T b, T c) {
  if constexpr (std::is_same_v<T, float>) return fmaf(a, b, c);
  else return fma(a, b, c);
}

// ---------------------------------------------------------------------------
// signed-permutation codes of fixed rotations
// code = p0 | p1 << 2 | p2 << 4 | n0 << 6 | n1 << 7 | n2 << 8: column k of the
// rotation is (-1)^{n_k} e_{p_k}.  -1 = generic dense rotation.
// ---------------------------------------------------------------------------
constexpr int XR_GENERIC = -1;
__host__ __device__ constexpr int xr_code(int p0, int p1, int p2, int n0, int n1, int n2) {
  return p0 | (p1 << 2) | (p2 << 4) | (n0 << 6) | (n1 << 7) | (n2 << 8);
}
__host__ __device__ constexpr int xr_perm(int code, int k) { return (code >> (2 * k)) & 3; }
__host__ __device__ constexpr bool xr_neg(int code, int k) { return (code >> (6 + k)) & 1; }
constexpr int XR_IDENTITY = xr_code(0, 1, 2, 0, 0, 0);
constexpr int XR_RX_PLUS = xr_code(0, 2, 1, 0, 0, 1);   // Rx(+pi/2): e1 -> e2, e2 -> -e1
constexpr int XR_RX_MINUS = xr_code(0, 2, 1, 0, 1, 0);  // Rx(-pi/2): e1 -> -e2, e2 -> e1
constexpr int XR_TO_X = xr_code(2, 1, 0, 1, 0, 0);      // z -> x: [[0,0,1],[0,1,0],[-1,0,0]]
constexpr int XR_TO_Y = xr_code(0, 2, 1, 0, 1, 0);      // z -> y: [[1,0,0],[0,0,1],[0,-1,0]]

// Column k of R (row-major 3x3) as a 3-vector.
template <typename T>
struct V3 {
  T x, y, z;
};
template <typename T>
__device__ __forceinline__ V3<T> col(const T (&R)[9], int k) {
  return {R[k], R[3 + k], R[6 + k]};
}
template <typename T>
__device__ __forceinline__ V3<T> neg_if(V3<T> v, bool n) {
  return n ? V3<T>{-v.x, -v.y, -v.z} : v;
}
template <typename T>
__device__ __forceinline__ void set_col(T (&R)[9], int k, V3<T> v) {
  R[k] = v.x;
  R[3 + k] = v.y;
  R[6 + k] = v.z;
}
template <typename T>
__device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
  return {fma_(a.y, b.z, -(a.z * b.y)), fma_(a.z, b.x, -(a.x * b.z)), fma_(a.x, b.y, -(a.y * b.x))};
}
template <typename T>
__device__ __forceinline__ T dot(V3<T> a, V3<T> b) {
  return fma_(a.x, b.x, fma_(a.y, b.y, a.z * b.z));
}
template <typename T>
__device__ __forceinline__ V3<T> sub(V3<T> a, V3<T> b) {
  return {a.x - b.x, a.y - b.y, a.z - b.z};
}
// R v and R^T v for row-major 3x3 (first 9 of a 3x4 with stride 4 handled by callers)
template <typename T>
__device__ __forceinline__ V3<T> mulv(const T (&R)[9], V3<T> v) {
  return {fma_(R[0], v.x, fma_(R[1], v.y, R[2] * v.z)), fma_(R[3], v.x, fma_(R[4], v.y, R[5] * v.z)),
          fma_(R[6], v.x, fma_(R[7], v.y, R[8] * v.z))};
}
template <typename T>
__device__ __forceinline__ V3<T> mulvt(const T (&R)[9], V3<T> v) {
  return {fma_(R[0], v.x, fma_(R[3], v.y, R[6] * v.z)), fma_(R[1], v.x, fma_(R[4], v.y, R[7] * v.z)),
          fma_(R[2], v.x, fma_(R[5], v.y, R[8] * v.z))};
}
// C = A B for 3x3
template <typename T>
__device__ __forceinline__ void mul33(const T (&A)[9], const T (&B)[9], T (&C)[9]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      C[r * 3 + c] = fma_(A[r * 3], B[c], fma_(A[r * 3 + 1], B[3 + c], A[r * 3 + 2] * B[6 + c]));
}
// C = A^T B
template <typename T>
__device__ __forceinline__ void mul33tn(const T (&A)[9], const T (&B)[9], T (&C)[9]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) C[r * 3 + c] = fma_(A[r], B[c], fma_(A[3 + r], B[3 + c], A[6 + r] * B[6 + c]));
}

// Pose = rotation + translation
template <typename T>
struct PoseT {
  T R[9];
  V3<T> p;
};

// Load the rotation / translation of a 3x4 from model memory.
template <typename T>
__device__ __forceinline__ void load_R(const T *X, T (&R)[9]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) R[r * 3 + c] = X[r * 4 + c];
}
template <typename T>
__device__ __forceinline__ V3<T> load_p(const T *X) {
  return {X[3], X[7], X[11]};
}

// Rp = Rparent * Xrot for a fixed rotation given by code (or dense from X).
template <int CODE, typename T>
__device__ __forceinline__ void apply_xrot(const T (&Rpar)[9], const T *X, T (&Rout)[9]) {
  if constexpr (CODE == XR_GENERIC) {
    T XR[9];
    load_R(X, XR);
    mul33(Rpar, XR, Rout);
  } else {
    set_col(Rout, 0, neg_if(col(Rpar, xr_perm(CODE, 0)), xr_neg(CODE, 0)));
    set_col(Rout, 1, neg_if(col(Rpar, xr_perm(CODE, 1)), xr_neg(CODE, 1)));
    set_col(Rout, 2, neg_if(col(Rpar, xr_perm(CODE, 2)), xr_neg(CODE, 2)));
  }
}
// Rotation of a root joint: the fixed rotation itself.
template <int CODE, typename T>
__device__ __forceinline__ void root_xrot(const T *X, T (&Rout)[9]) {
  if constexpr (CODE == XR_GENERIC) {
    load_R(X, Rout);
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) Rout[i] = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) Rout[xr_perm(CODE, k) * 3 + k] = xr_neg(CODE, k) ? T(-1) : T(1);
  }
}
// p + R * t with t's structurally-zero components skipped (MASK bit i: t_i may be nonzero).
template <int MASK, typename T>
__device__ __forceinline__ V3<T> add_rot_t(V3<T> p, const T (&R)[9], V3<T> t) {
  V3<T> out = p;
  if constexpr (MASK & 1) out = {fma_(R[0], t.x, out.x), fma_(R[3], t.x, out.y), fma_(R[6], t.x, out.z)};
  if constexpr (MASK & 2) out = {fma_(R[1], t.y, out.x), fma_(R[4], t.y, out.y), fma_(R[7], t.y, out.z)};
  if constexpr (MASK & 4) out = {fma_(R[2], t.z, out.x), fma_(R[5], t.z, out.y), fma_(R[8], t.z, out.z)};
  return out;
}

// ---------------------------------------------------------------------------
// Problem-class helpers (constexpr over the topology)
// ---------------------------------------------------------------------------
template <class P>
__host__ __device__ constexpr bool is_anc(int j, int link) {
  for (int l = link; l >= 0; l = P::parent(l))
    if (l == j) return true;
  return false;
}
__host__ __device__ constexpr int cdim(int kind) {
  return (kind == K_SPHERE || kind == K_PLANE || kind == K_DIST)             ? 1
         : (kind == K_POSE || kind == K_REL || kind == K_PBND)               ? 6
                                                                             : 2;  // AXIS, COM, LINE, HULL
}
// Model slot of constraint c: a sub-problem (one constraint of a stack, used
// by the cyclic form) reads the slot of the constraint it stands for.
template <class P, class = void>
struct CBase {
  static constexpr int value = 0;
};
template <class P>
struct CBase<P, std::void_t<decltype(P::CBASE)>> {
  static constexpr int value = P::CBASE;
};
// Constraint C of the stack P alone (same robot, one constraint): the unit of
// one step of the cyclic getDescentStep (Sec. IV-C).
template <class P, int C>
struct Sub : P {
  static constexpr int NC = 1;
  static constexpr int CBASE = C;
  __host__ __device__ static constexpr int ckind(int) { return P::ckind(C); }
  __host__ __device__ static constexpr int cfa(int) { return P::cfa(C); }
  __host__ __device__ static constexpr int cfb(int) { return P::cfb(C); }
};
template <class P>
__host__ __device__ constexpr int roff(int c) {
  int r = 0;
  for (int i = 0; i < c; ++i) r += cdim(P::ckind(i));
  return r;
}
template <class P>
__host__ __device__ constexpr int kdim() {
  return roff<P>(P::NC);
}
template <class P>
__host__ __device__ constexpr bool needs_pos() {  // any constraint uses translations
  for (int c = 0; c < P::NC; ++c)
    if (P::ckind(c) != K_SPHERE && P::ckind(c) != K_AXIS) return true;
  return false;
}
template <class P>
__host__ __device__ constexpr bool needs_fk() {
  for (int c = 0; c < P::NC; ++c)
    if (P::ckind(c) != K_SPHERE) return true;
  return false;
}
template <class P>
__host__ __device__ constexpr bool needs_com() {
  for (int c = 0; c < P::NC; ++c)
    if (P::ckind(c) == K_COM || P::ckind(c) == K_HULL) return true;
  return false;
}
// Sign with which joint j enters row block of constraint c (0 = structurally zero).
template <class P>
__host__ __device__ constexpr int col_sign(int c, int j) {
  const int k = P::ckind(c);
  if (k == K_SPHERE || k == K_COM || k == K_HULL) return 1;
  if (k == K_REL || k == K_DIST)
    return (is_anc<P>(j, P::frame_link(P::cfb(c))) ? 1 : 0) - (is_anc<P>(j, P::frame_link(P::cfa(c))) ? 1 : 0);
  return is_anc<P>(j, P::frame_link(P::cfa(c))) ? 1 : 0;
}
// Structural nonzero of J[row][j].
template <class P>
__host__ __device__ constexpr bool jnz(int row, int j) {
  int c = 0;
  while (c + 1 < P::NC && roff<P>(c + 1) <= row) ++c;
  const int k = P::ckind(c), rr = row - roff<P>(c);
  const int s = col_sign<P>(c, j);
  if (s == 0) return false;
  if (k == K_AXIS) return P::jtype(j) == REV;
  if ((k == K_POSE || k == K_REL || k == K_PBND) && rr >= 3) return P::jtype(j) == REV;
  return true;
}

// ---------------------------------------------------------------------------
// Forward kinematics over the compile-time topology.
// ---------------------------------------------------------------------------
template <class P, typename T>
struct Kin {
  T R[P::D][9];       // world rotation of joint frame j after its motion
  V3<T> p[P::D];      // world origin of joint frame j
  V3<T> z[P::D];      // world axis of joint j
  T fR[P::NF > 0 ? P::NF : 1][9];
  V3<T> fp[P::NF > 0 ? P::NF : 1];
  V3<T> mc;           // sum_j m_j c_j (accumulated during FK when a CoM constraint is present)
};

struct NoVisit {
  template <class J, class R, class V>
  __device__ __forceinline__ void operator()(J, const R &, V) const {}
};
struct NoStop {
  __device__ __forceinline__ bool operator()() const { return false; }
};

// World transforms of every joint frame (and the task frames).  The model m
// is a ModelT or any view with rows X[j] and fX[f] (and mass / com where a
// CoM constraint needs them).  `visit(j, R_j,
// p_j)` is called right after joint j is placed, and joints after `stop()`
// becomes true are skipped, so consumers can use each link's pose while it is
// live (the collision check does) instead of keeping the whole tree.
// COM: accumulate the mass moment sum_j m_j c_j (its x and y, all that the
// CoM constraints read) for problems with a CoM constraint; the collision
// check, which only needs the link poses, leaves it out.
template <class P, bool POS, bool COM, class Ops, typename T, class Visit, class Stop, class M>
__device__ __forceinline__ void fk_impl(const Ops &ops, const M &m, const T (&q)[P::D], Kin<P, T> &k,
                                        const Visit &visit, const Stop &stop) {
  static_for<P::D>([&](auto JJ) {
    constexpr int j = decltype(JJ)::value;
    if (stop()) return;
    constexpr int pa = P::parent(j);
    constexpr int code = P::xrot(j);
    T Rpre[9];
    [[maybe_unused]] V3<T> ppre{T(0), T(0), T(0)};  // unused without positions
    if constexpr (pa < 0) {
      root_xrot<code>(m.X[j], Rpre);
      if constexpr (POS) ppre = load_p(m.X[j]);
    } else {
      apply_xrot<code>(k.R[pa], m.X[j], Rpre);
      if constexpr (POS) ppre = add_rot_t<P::xtmask(j)>(k.p[pa], k.R[pa], load_p(m.X[j]));
    }
    k.z[j] = col(Rpre, 2);
    if constexpr (j == 0 && COM) k.mc = V3<T>{T(0), T(0), T(0)};
    if constexpr (P::jtype(j) == REV) {
      T s, c;
      ops.sincos(q[j], s, c);
      V3<T> c0 = col(Rpre, 0), c1 = col(Rpre, 1);
      set_col(k.R[j], 0, V3<T>{fma_(c, c0.x, s * c1.x), fma_(c, c0.y, s * c1.y), fma_(c, c0.z, s * c1.z)});
      set_col(k.R[j], 1, V3<T>{fma_(c, c1.x, -(s * c0.x)), fma_(c, c1.y, -(s * c0.y)), fma_(c, c1.z, -(s * c0.z))});
      set_col(k.R[j], 2, col(Rpre, 2));
      if constexpr (POS) k.p[j] = ppre;
    } else {
#pragma unroll
      for (int i = 0; i < 9; ++i) k.R[j][i] = Rpre[i];
      if constexpr (POS) k.p[j] = {fma_(q[j], Rpre[2], ppre.x), fma_(q[j], Rpre[5], ppre.y), fma_(q[j], Rpre[8], ppre.z)};
    }
    if constexpr (COM) {  // x and y of c_j = p_j + R_j com_j (the order of add_rot_t)
      const T cx = fma_(k.R[j][2], m.com[j][2], fma_(k.R[j][1], m.com[j][1], fma_(k.R[j][0], m.com[j][0], k.p[j].x)));
      const T cy = fma_(k.R[j][5], m.com[j][2], fma_(k.R[j][4], m.com[j][1], fma_(k.R[j][3], m.com[j][0], k.p[j].y)));
      k.mc = {fma_(m.mass[j], cx, k.mc.x), fma_(m.mass[j], cy, k.mc.y), T(0)};
    }
    visit(JJ, k.R[j], k.p[j]);
  });
  if (stop()) return;
  static_for<P::NF>([&](auto FF) {
    constexpr int f = decltype(FF)::value;
    constexpr int l = P::frame_link(f);
    apply_xrot<P::frot(f)>(k.R[l], m.fX[f], k.fR[f]);
    if constexpr (POS) k.fp[f] = add_rot_t<P::ftmask(f)>(k.p[l], k.R[l], load_p(m.fX[f]));
  });
}
template <class P, bool POS, class Ops, typename T, class Visit = NoVisit, class Stop = NoStop, class M = ModelT<T>>
__device__ __forceinline__ void fk(const Ops &ops, const M &m, const T (&q)[P::D], Kin<P, T> &k,
                                   const Visit &visit = Visit{}, const Stop &stop = Stop{}) {
  fk_impl<P, POS, POS && needs_com<P>(), Ops, T, Visit, Stop, M>(ops, m, q, k, visit, stop);
}
// Link poses only (no mass moment): the collision check.
template <class P, class Ops, typename T, class Visit, class Stop, class M = ModelT<T>>
__device__ __forceinline__ void fk_links(const Ops &ops, const M &m, const T (&q)[P::D], Kin<P, T> &k,
                                         const Visit &visit, const Stop &stop) {
  fk_impl<P, true, false, Ops, T, Visit, Stop, M>(ops, m, q, k, visit, stop);
}

// ---------------------------------------------------------------------------
// SO(3) log map (Sec. IV-A) and the inverse left Jacobian.
// theta = atan2(|w|, (tr R - 1)/2), w = vee(R - R^T)/2.  theta < 1e-3: factor
// theta/sin(theta) -> 1 + theta^2/6 (the Taylor fallback of sinc); theta >
// 3pi/4: axis from the symmetric part, sign from w.
// ---------------------------------------------------------------------------
template <class Ops, typename T>
struct LogOut {
  V3<T> phi;
  T theta, s, c;  // theta, sin theta (= |w|), cos theta
};

template <class Ops, typename T>
__device__ __forceinline__ LogOut<Ops, T> so3_log(const T (&R)[9]) {
  LogOut<Ops, T> o;
  V3<T> w{T(0.5) * (R[7] - R[5]), T(0.5) * (R[2] - R[6]), T(0.5) * (R[3] - R[1])};
  T c = T(0.5) * (R[0] + R[4] + R[8] - T(1));
  T s2 = dot(w, w);
  T s = Ops::sqrt_(s2);
  o.s = s;
  o.c = c;
  if (c > T(0) && s < T(1e-3)) {
    // small angle: theta = asin(s) = s f(s), f = 1 + s^2/6 + 3 s^4/40 (next
    // term 5 s^6/112 < 1e-19), and phi = (theta / sin theta) w = f w: no atan2
    // (the acceptance of a converged configuration always lands here)
    T f = fma_(s2, fma_(s2, T(3.0 / 40.0), T(1.0 / 6.0)), T(1));
    o.theta = f * s;
    o.phi = {f * w.x, f * w.y, f * w.z};
    return o;
  }
  T th = Ops::atan2_(s, c);
  o.theta = th;
  if (th < T(1e-3)) {
    T f = fma_(th * th, T(1.0 / 6.0), T(1));
    o.phi = {f * w.x, f * w.y, f * w.z};
  } else if (th <= T(2.356194490192345)) {
    T f = th / s;
    o.phi = {f * w.x, f * w.y, f * w.z};
  } else {
    T S[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) S[r * 3 + cc] = T(0.5) * (R[r * 3 + cc] + R[cc * 3 + r]);
    // the axis from column i of S, i the largest diagonal entry; the
    // column is selected by value (no runtime index into a local array)
    const bool i1 = S[4] > S[0];
    const T d01 = i1 ? S[4] : S[0];
    const bool i2 = S[8] > d01;
    const T sii = i2 ? S[8] : d01;
    const T s0i = i2 ? S[2] : (i1 ? S[1] : S[0]);
    const T s1i = i2 ? S[5] : (i1 ? S[4] : S[3]);
    const T s2i = i2 ? S[8] : (i1 ? S[7] : S[6]);
    T omc = T(1) - c;
    T ai = Ops::sqrt_((sii - c) / omc);
    T inv = T(1) / (omc * ai);
    V3<T> a{(s0i - (!i1 && !i2 ? c : T(0))) * inv, (s1i - (i1 && !i2 ? c : T(0))) * inv,
            (s2i - (i2 ? c : T(0))) * inv};
    if (dot(a, w) < T(0)) a = {-a.x, -a.y, -a.z};
    o.phi = {th * a.x, th * a.y, th * a.z};
  }
  return o;
}

// Jl^{-1}(phi) v = v - 1/2 phi x v + beta phi x (phi x v),
// beta = 1/theta^2 - sin(theta) / (2 theta (1 - cos(theta))), series 1/12 + theta^2/720 + theta^4/30240
// below SMALL (0.3 in FP32, 1e-2 in FP64: where the closed form loses accuracy to cancellation).
template <typename T>
__device__ __forceinline__ T jl_inv_beta(T th, T s, T c) {
  constexpr T SMALL = std::is_same_v<T, float> ? T(0.3) : T(1e-2);
  T th2 = th * th;
  if (th < SMALL) return fma_(th2, fma_(th2, T(1.0 / 30240.0), T(1.0 / 720.0)), T(1.0 / 12.0));
  T omc = (c > T(0)) ? (s * s) / (T(1) + c) : (T(1) - c);
  return T(1) / th2 - s / (T(2) * th * omc);
}
template <typename T>
__device__ __forceinline__ V3<T> jl_inv_apply(V3<T> phi, T beta, V3<T> v) {
  V3<T> a = cross(phi, v);
  V3<T> b = cross(phi, a);
  return {fma_(beta, b.x, fma_(T(-0.5), a.x, v.x)), fma_(beta, b.y, fma_(T(-0.5), a.y, v.y)),
          fma_(beta, b.z, fma_(T(-0.5), a.z, v.z))};
}

// ---------------------------------------------------------------------------
// Cholesky of a K x K SPD matrix held as the lower triangle A[i*(i+1)/2 + j],
// in place (Dahlquist & Bjorck, no pivoting), and the solves L L^T x = b.
// The factorisation returns the smallest pre-square-root pivot.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// Factorisation only: A is overwritten by L (lower triangle), inv[j] = 1 / L_jj.
template <int K, class Ops, typename T>
__device__ __forceinline__ T cholesky_factor(T (&A)[K * (K + 1) / 2], T (&inv)[K]) {
  T minpiv = T(1e30);
#pragma unroll
  for (int j = 0; j < K; ++j) {
    T s = A[tri(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) s = fma_(-A[tri(j, k)], A[tri(j, k)], s);
    minpiv = s < minpiv ? s : minpiv;
    T ij = Ops::rsqrt_(s);
    inv[j] = ij;
    A[tri(j, j)] = s * ij;
#pragma unroll
    for (int i = j + 1; i < K; ++i) {
      T t = A[tri(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) t = fma_(-A[tri(i, k)], A[tri(j, k)], t);
      A[tri(i, j)] = t * ij;
    }
  }
  return minpiv;
}

// b <- (L L^T)^{-1} b with the factor from cholesky_factor.
template <int K, typename T>
__device__ __forceinline__ void cholesky_subst(const T (&L)[K * (K + 1) / 2], const T (&inv)[K], T (&b)[K]) {
#pragma unroll
  for (int i = 0; i < K; ++i) {
    T s = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s = fma_(-L[tri(i, k)], b[k], s);
    b[i] = s * inv[i];
  }
#pragma unroll
  for (int i = K - 1; i >= 0; --i) {
    T s = b[i];
#pragma unroll
    for (int k = i + 1; k < K; ++k) s = fma_(-L[tri(k, i)], b[k], s);
    b[i] = s * inv[i];
  }
}

template <int K, class Ops, typename T>
__device__ __forceinline__ T cholesky_solve(T (&A)[K * (K + 1) / 2], T (&b)[K]) {
  T inv[K];
  const T minpiv = cholesky_factor<K, Ops>(A, inv);
  cholesky_subst<K>(A, inv, b);
  return minpiv;
}


// Nearest point of a convex polygon (vertices v[2 nv], counter-clockwise) to
// the point (x, y).  mode 0: inside (the point itself); 1: on an edge's
// interior, (nx, ny) its outward unit normal; 2: at a vertex.  Ties between
// edges go to the first.
template <typename T>
__device__ __forceinline__ int polygon_nearest(const T *v, int nv, T x, T y, T &px, T &py, T &nx, T &ny) {
  bool inside = true;
  for (int e = 0; e < nv; ++e) {
    const int f = e + 1 < nv ? e + 1 : 0;
    const T cr = (v[2 * f] - v[2 * e]) * (y - v[2 * e + 1]) - (v[2 * f + 1] - v[2 * e + 1]) * (x - v[2 * e]);
    if (cr < T(0)) inside = false;
  }
  px = x;
  py = y;
  nx = ny = T(0);
  if (inside) return 0;
  int mode = 2;
  T best = T(0);
  bool first = true;
  for (int e = 0; e < nv; ++e) {
    const int f = e + 1 < nv ? e + 1 : 0;
    const T ex = v[2 * f] - v[2 * e], ey = v[2 * f + 1] - v[2 * e + 1];
    T t = ((x - v[2 * e]) * ex + (y - v[2 * e + 1]) * ey) / (ex * ex + ey * ey);
    const bool interior = t > T(0) && t < T(1);
    t = t < T(0) ? T(0) : (t > T(1) ? T(1) : t);
    const T qx = v[2 * e] + t * ex, qy = v[2 * e + 1] + t * ey;
    const T dd = (x - qx) * (x - qx) + (y - qy) * (y - qy);
    if (first || dd < best) {
      first = false;
      best = dd;
      px = qx;
      py = qy;
      mode = interior ? 1 : 2;
      const T el = sqrt(ex * ex + ey * ey);
      nx = ey / el;
      ny = -ex / el;
    }
  }
  return mode;
}

}  // namespace mcp
