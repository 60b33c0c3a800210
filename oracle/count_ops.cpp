/*
 * Operation-counting build of the FP64 oracle (mcp_oracle.c).
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE ONLY: the benchmark's roofline and the
 * tests use it to count the arithmetic the method performs; the product path
 * never loads it.
 *
 * The oracle's source is compiled unchanged, as C++, with every `double`
 * replaced by `Counted`, a wrapper of one double (same size and layout, so
 * the caller's arrays are shared as they are) whose operators perform the
 * FP64 operation and tally it.  The count follows the straight-line code a
 * tracing compiler emits for a fixed robot and constraint stack (Sec. IV-A,
 * "Tracing Compiler for Constraints": structural zeros and constant folding
 * are resolved at trace time), so operations whose result is fixed by an
 * operand's value are free:
 *   x * 0, x * 1, x * -1, x + 0, x - 0, 0 - x, x / 1, x / -1 and negation
 *   are not counted (they are exact in floating point and a traced program
 *   folds the structural zeros and signed unit entries away);
 *   every other +, -, * and / counts 1 flop (the oracle forms a*b + c as two
 *   operations, an FMA counts 2);
 *   sqrt, sin, cos and atan2 are counted apart (special-function work, not
 *   flops); comparisons, fabs, fmin and fmax are free.
 * A value that is exactly zero or one by accident (not structurally) is
 * treated the same way; with continuous random inputs that has probability
 * zero.
 *
 * Counting is per thread; the exported counters are read after a
 * single-threaded call.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

namespace {
struct OpTally {
  uint64_t add, mul, div, sqrt, trig, atan2;
};
thread_local OpTally g_tally;
}  // namespace

struct Counted {
  double v;
  Counted() = default;
  constexpr Counted(double x) : v(x) {}
  explicit operator double() const { return v; }
  explicit operator int() const { return static_cast<int>(v); }
  Counted &operator+=(Counted o);
  Counted &operator-=(Counted o);
  Counted &operator*=(Counted o);
  Counted &operator/=(Counted o);
};
static_assert(sizeof(Counted) == sizeof(double), "Counted must alias double arrays");

static inline bool unit(double x) { return x == 1.0 || x == -1.0; }

inline Counted operator+(Counted a, Counted b) {
  if (a.v != 0.0 && b.v != 0.0) ++g_tally.add;
  return Counted(a.v + b.v);
}
inline Counted operator-(Counted a, Counted b) {
  if (a.v != 0.0 && b.v != 0.0) ++g_tally.add;
  return Counted(a.v - b.v);
}
inline Counted operator*(Counted a, Counted b) {
  if (a.v != 0.0 && b.v != 0.0 && !unit(a.v) && !unit(b.v)) ++g_tally.mul;
  return Counted(a.v * b.v);
}
inline Counted operator/(Counted a, Counted b) {
  if (a.v != 0.0 && !unit(b.v)) ++g_tally.div;
  return Counted(a.v / b.v);
}
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline Counted operator+(Counted a) { return a; }
inline Counted &Counted::operator+=(Counted o) { return *this = *this + o; }
inline Counted &Counted::operator-=(Counted o) { return *this = *this - o; }
inline Counted &Counted::operator*=(Counted o) { return *this = *this * o; }
inline Counted &Counted::operator/=(Counted o) { return *this = *this / o; }
inline bool operator<(Counted a, Counted b) { return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { return a.v >= b.v; }
inline bool operator==(Counted a, Counted b) { return a.v == b.v; }
inline bool operator!=(Counted a, Counted b) { return a.v != b.v; }

inline Counted sqrt(Counted a) {
  ++g_tally.sqrt;
  return Counted(::sqrt(a.v));
}
inline Counted sin(Counted a) {
  ++g_tally.trig;
  return Counted(::sin(a.v));
}
inline Counted cos(Counted a) {
  ++g_tally.trig;
  return Counted(::cos(a.v));
}
inline Counted atan2(Counted y, Counted x) {
  ++g_tally.atan2;
  return Counted(::atan2(y.v, x.v));
}
inline Counted fabs(Counted a) { return Counted(::fabs(a.v)); }
inline Counted fmax(Counted a, Counted b) { return Counted(::fmax(a.v, b.v)); }
inline Counted fmin(Counted a, Counted b) { return Counted(::fmin(a.v, b.v)); }
inline bool isfinite(Counted a) { return std::isfinite(a.v); }

#define double Counted
extern "C" {
#include "mcp_oracle.c"
}
#undef double

/* Per configuration of a batch (SoA [d * ld]), the operations of
 *   out[i][0..5]:  one evaluation of the stacked residual F (forward
 *                  kinematics and every constraint), as the convergence test
 *                  and the acceptance take it;
 *   out[i][6..11]: one LM step: F and J together, the descent step of
 *                  getDescentStep (Gram matrix, Cholesky, solves, J^T y) and
 *                  the update q - dq;
 *   out[i][12..17]: one VJP g - J^T (J J^T)^{-1} J g at the configuration;
 * each as (add, mul, div, sqrt, sin/cos, atan2).  Single-threaded. */
extern "C" void oc_count(const or_robot *rb, const or_constraint *cons, int nc, const or_params *p, int64_t n,
                         int64_t ld, const double *q_in, const double *g_in, uint64_t *out) {
  const int d = rb->nj;
  int k = 0;
  for (int i = 0; i < nc; ++i) k += cons_dim(cons[i].kind);
  for (int64_t i = 0; i < n; ++i) {
    Counted q[OR_MAXJ], F[OR_MAXK], dq[OR_MAXJ], g[OR_MAXJ], v[OR_MAXJ];
    static Counted J[OR_MAXK * OR_MAXJ];
    for (int j = 0; j < d; ++j) {
      q[j] = Counted(q_in[j * ld + i]);
      g[j] = Counted(g_in ? g_in[j * ld + i] : 0.0);
    }
    uint64_t *o = out + i * 18;
    g_tally = OpTally{};
    eval_stack(rb, cons, 0, nc, q, F, NULL);
    const OpTally e = g_tally;
    g_tally = OpTally{};
    memset(J, 0, sizeof(Counted) * k * d);
    eval_stack(rb, cons, 0, nc, q, F, J);
    descent(p, k, d, J, F, dq);
    for (int j = 0; j < d; ++j) q[j] = q[j] - dq[j];
    const OpTally s = g_tally;
    for (int j = 0; j < d; ++j) q[j] = Counted(q_in[j * ld + i]);
    g_tally = OpTally{};
    vjp_one(rb, cons, nc, q, g, v);
    const OpTally w = g_tally;
    const OpTally *t[3] = {&e, &s, &w};
    for (int m = 0; m < 3; ++m) {
      o[6 * m + 0] = t[m]->add;
      o[6 * m + 1] = t[m]->mul;
      o[6 * m + 2] = t[m]->div;
      o[6 * m + 3] = t[m]->sqrt;
      o[6 * m + 4] = t[m]->trig;
      o[6 * m + 5] = t[m]->atan2;
    }
  }
}
