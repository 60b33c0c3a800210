// Problem classes: compile-time robot structure + stacked constraint kinds.
//
// Each class plays the role of one traced robot/constraint pair of the paper's
// tracing compiler (Sec. IV-A; Sec. VI: constraints are known a priori).  A
// loaded robot is bound to a class only if its topology, joint types, the
// structural zeros of its fixed offsets and its constraint kinds/frames match
// exactly (checked on the host when loading); numeric values (link lengths,
// masses, references, ...) are runtime data.
#pragma once

#include "mcp_device.cuh"

namespace mcp {

// --- a point in R^3 as a Cartesian robot (prismatic x, y, z); F = |q| - r ---
struct ProbSphere3 {
  static constexpr const char *name = "sphere3";
  static constexpr int D = 3, NF = 1, NC = 1;
  __host__ __device__ static constexpr int parent(int j) { return j - 1; }
  __host__ __device__ static constexpr int jtype(int) { return PRIS; }
  __host__ __device__ static constexpr int xrot(int j) {
    constexpr int a[3] = {70, 18, 280};
    return a[j];
  }
  __host__ __device__ static constexpr int xtmask(int) { return 0; }
  __host__ __device__ static constexpr int frame_link(int) { return 2; }
  __host__ __device__ static constexpr int frot(int) { return XR_IDENTITY; }
  __host__ __device__ static constexpr int ftmask(int) { return 0; }
  __host__ __device__ static constexpr int ckind(int) { return K_SPHERE; }
  __host__ __device__ static constexpr int cfa(int) { return -1; }
  __host__ __device__ static constexpr int cfb(int) { return -1; }
};

// --- the Cartesian point on four planes through one point (k = 4 > d = 3): a
//     consistent overdetermined stack, where J J^T is singular and the outer
//     form (J^T J + lambda I)^-1 J^T F of Alg. 2 is the step that works ---
struct ProbPoint3Planes4 : ProbSphere3 {
  static constexpr const char *name = "point3_planes4";
  static constexpr int NC = 4;
  __host__ __device__ static constexpr int ckind(int) { return K_PLANE; }
  __host__ __device__ static constexpr int cfa(int) { return 0; }
};

// --- 7-DoF DH chain: a = 0, d_i along z, twists alternating +-pi/2 ---
struct ArmChain7 {
  __host__ __device__ static constexpr int arm_xrot(int i) {
    return i == 0 ? XR_IDENTITY : (i % 2 == 1 ? XR_RX_PLUS : XR_RX_MINUS);
  }
};

struct ProbArm7Axis : ArmChain7 {  // end-effector z parallel to world z (k = 2)
  static constexpr const char *name = "arm7_axis";
  static constexpr int D = 7, NF = 1, NC = 1;
  __host__ __device__ static constexpr int parent(int j) { return j - 1; }
  __host__ __device__ static constexpr int jtype(int) { return REV; }
  __host__ __device__ static constexpr int xrot(int j) { return arm_xrot(j); }
  __host__ __device__ static constexpr int xtmask(int j) { return j == 0 ? 7 : 4; }
  __host__ __device__ static constexpr int frame_link(int) { return 6; }
  __host__ __device__ static constexpr int frot(int) { return XR_IDENTITY; }
  __host__ __device__ static constexpr int ftmask(int) { return 4; }
  __host__ __device__ static constexpr int ckind(int) { return K_AXIS; }
  __host__ __device__ static constexpr int cfa(int) { return 0; }
  __host__ __device__ static constexpr int cfb(int) { return -1; }
};

struct ProbArm7Pose : ProbArm7Axis {  // full 6-D end-effector TSR, Eq. 1 (k = 6)
  static constexpr const char *name = "arm7_pose";
  __host__ __device__ static constexpr int ckind(int) { return K_POSE; }
};

// --- task constraints on the 7-DoF arm (Sec. III: a tool held level on a
//     table, a peg inserted along a vertical line; Sec. II: a bounded TSR) ---
struct ProbArm7Tray : ProbArm7Axis {  // EE on a plane + EE z vertical (k = 3, two constraints)
  static constexpr const char *name = "arm7_tray";
  static constexpr int NC = 2;
  __host__ __device__ static constexpr int ckind(int c) { return c == 0 ? K_PLANE : K_AXIS; }
};
struct ProbArm7Peg : ProbArm7Axis {  // EE on a line + EE z vertical (k = 4, two constraints)
  static constexpr const char *name = "arm7_peg";
  static constexpr int NC = 2;
  __host__ __device__ static constexpr int ckind(int c) { return c == 0 ? K_LINE : K_AXIS; }
};
struct ProbArm7Tsr : ProbArm7Axis {  // bounded TSR, Eq. 1 with B^w (k = 6)
  static constexpr const char *name = "arm7_tsr";
  __host__ __device__ static constexpr int ckind(int) { return K_PBND; }
};

// --- two copies of the 7-DoF chain, bases offset; relative EE pose (Eq. 2) ---
struct ProbDual14Rel : ArmChain7 {
  static constexpr const char *name = "dual14_rel";
  static constexpr int D = 14, NF = 2, NC = 1;
  __host__ __device__ static constexpr int parent(int j) { return (j == 0 || j == 7) ? -1 : j - 1; }
  __host__ __device__ static constexpr int jtype(int) { return REV; }
  __host__ __device__ static constexpr int xrot(int j) { return arm_xrot(j % 7); }
  __host__ __device__ static constexpr int xtmask(int j) { return (j % 7) == 0 ? 7 : 4; }
  __host__ __device__ static constexpr int frame_link(int f) { return f == 0 ? 6 : 13; }
  __host__ __device__ static constexpr int frot(int) { return XR_IDENTITY; }
  __host__ __device__ static constexpr int ftmask(int) { return 4; }
  __host__ __device__ static constexpr int ckind(int) { return K_REL; }
  __host__ __device__ static constexpr int cfa(int) { return 0; }
  __host__ __device__ static constexpr int cfb(int) { return 1; }
};

// --- the dual arm carrying a rod on a table: fixed EE distance (closed
//     linkage) and both EEs on a plane (k = 3, three constraints) ---
struct ProbDual14Rod : ProbDual14Rel {
  static constexpr const char *name = "dual14_rod";
  static constexpr int NC = 3;
  __host__ __device__ static constexpr int ckind(int c) { return c == 0 ? K_DIST : K_PLANE; }
  __host__ __device__ static constexpr int cfa(int c) { return c == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int cfb(int c) { return c == 0 ? 1 : -1; }
};

// --- 36-DoF humanoid tree: base (3P + 3R), two 6-DoF legs, 2 + 2 torso/neck,
//     two 7-DoF arms; feet TSRs (Eq. 1), hands relative pose (Eq. 2), CoM xy ---
struct ProbHumanoid36 {
  static constexpr const char *name = "humanoid36";
  static constexpr int D = 36, NF = 4, NC = 4;
  __host__ __device__ static constexpr int parent(int j) {
    constexpr int a[36] = {-1, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 5, 12, 13, 14, 15, 16,
                           5, 18, 19, 20, 19, 22, 23, 24, 25, 26, 27, 19, 29, 30, 31, 32, 33, 34};
    return a[j];
  }
  __host__ __device__ static constexpr int jtype(int j) { return j < 3 ? PRIS : REV; }
  __host__ __device__ static constexpr int xrot(int j) {
    constexpr int a[36] = {70, 18, 280, 36, 152, 9, 262, 70, 18, 36, 36, 9, 262, 70, 18, 36, 36, 9,
                           262, 152, 280, 152, 36, 9, 262, 152, 280, 152, 9, 36, 9, 262, 152, 280, 152, 9};
    return a[j];
  }
  __host__ __device__ static constexpr int xtmask(int j) {
    constexpr int a[36] = {0, 0, 0, 0, 0, 0, 3, 4, 1, 2, 2, 0, 3, 4, 1, 2, 2, 0,
                           1, 4, 2, 4, 6, 4, 1, 4, 2, 0, 0, 6, 4, 1, 4, 2, 0, 0};
    return a[j];
  }
  __host__ __device__ static constexpr int frame_link(int f) {
    constexpr int a[4] = {11, 17, 28, 35};
    return a[f];
  }
  __host__ __device__ static constexpr int frot(int) { return 262; }
  __host__ __device__ static constexpr int ftmask(int f) { return f < 2 ? 5 : 1; }
  __host__ __device__ static constexpr int ckind(int c) {
    constexpr int a[4] = {K_POSE, K_POSE, K_REL, K_COM};
    return a[c];
  }
  __host__ __device__ static constexpr int cfa(int c) {
    constexpr int a[4] = {0, 1, 2, 0};
    return a[c];
  }
  __host__ __device__ static constexpr int cfb(int c) {
    constexpr int a[4] = {-1, -1, 3, 1};
    return a[c];
  }
};

// --- the humanoid with the CoM constraint as the distance to the support
//     polygon (zero inside) instead of equality to its centre ---
struct ProbHumanoid36Hull : ProbHumanoid36 {
  static constexpr const char *name = "humanoid36_hull";
  __host__ __device__ static constexpr int ckind(int c) { return c == 3 ? K_HULL : ProbHumanoid36::ckind(c); }
};

// Classes whose FP32 projection also has a two-lanes-per-configuration
// kernel (one lane per chain of a two-chain tree; the autotuner chooses).
template <class P>
__host__ __device__ constexpr bool has_pair_kernel() {
  return std::is_same_v<P, ProbDual14Rel>;
}

}  // namespace mcp
