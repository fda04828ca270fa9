// Operation tally of the sweep kernel's formulas (hgks_count_flops): the
// device closed forms of physics.cuh, recon.cuh, compat.cuh and the sweep's
// face-field and tangential passes, instantiated on the host with a counting
// number type, for ONE face and ONE face point -- the work the method needs
// per face, without the recomputation on a tile's halo.  This is the
// algorithmic count behind the sweep kernel's ALU roofline; it is formed from
// the formulas, not from the executed instructions of the kernel.
//
// Counting rules: an addition, subtraction, multiplication or division of
// two values one of which varies per face is one operation (a fused
// multiply-add is a multiplication and an addition); operations whose
// operands are all per-run constants (numerical literals, the gas constants,
// the time step) are folded, as the compiler folds or hoists them; x * 1,
// x * -1, x + 0 and x * 0 are free; an operation repeated on the same
// operands within one part is counted once (value numbering: common
// subexpressions are evaluated once, as an optimising compiler does, but
// nothing is reassociated); only operations that an output of the part
// depends on are counted (dead results -- e.g. the derivative of a
// tangential polynomial when only its values are used -- are not evaluated
// by the kernel either).  Square roots, exponentials, error functions and
// powers are tallied separately (not as flops).  Comparisons, negations and
// absolute values are free.
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <type_traits>
#include <vector>

#include "engine.h"
#include "sweep.cuh"

namespace hgks {

struct OpTally {
  long long add = 0, mul = 0, div = 0, sqrt = 0, exp = 0, erf = 0, pow = 0;
};

enum CntOp { OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_NEG, OP_SQRT, OP_EXP, OP_EXPM1, OP_ERF, OP_POW,
             OP_ABS };

// A number that tallies the operations done on it.  k: a per-run constant
// (identified by its value); otherwise id numbers the value.
struct Cnt {
  double v = 0.0;
  bool k = true;
  long long id = 0;
  __host__ __device__ inline Cnt() {}
  template <class U, class = typename std::enable_if<std::is_arithmetic<U>::value>::type>
  __host__ __device__ inline Cnt(U x) : v(double(x)), k(true), id(0) {}
};

// Host-side state of the tally: the value table of the current part and
// the expression graph (operation and operand value numbers of every value
// number; -1 for inputs), from which the operations the outputs depend on
// are counted.
struct TallyState {
  std::map<std::tuple<int, long long, long long, long long, long long>, long long> seen;
  std::vector<std::tuple<int, long long, long long>> node{std::make_tuple(-1, 0LL, 0LL)};
  long long next = 1;
};
static TallyState g_ts;

// Key of an operand: its value number, or the bits of a constant.
static inline std::pair<long long, long long> operand_key(const Cnt& a) {
  long long bits = 0;
  if (a.k) std::memcpy(&bits, &a.v, sizeof bits);
  return {a.k ? 0 : a.id, bits};
}

// Records op(a, b) = r (r.k false): counts it unless the same operation on
// the same operands was seen in this part, and gives r its value number.
[[maybe_unused]] static void record(int op, const Cnt& a, const Cnt& b, Cnt& r) {
  auto ka = operand_key(a), kb = operand_key(b);
  if ((op == OP_ADD || op == OP_MUL) && kb < ka) std::swap(ka, kb);  // commutative
  const auto key = std::make_tuple(op, ka.first, ka.second, kb.first, kb.second);
  auto it = g_ts.seen.find(key);
  if (it != g_ts.seen.end()) {
    r.id = it->second;
    return;
  }
  r.id = g_ts.next++;
  g_ts.seen.emplace(key, r.id);
  g_ts.node.emplace_back(op, a.k ? 0LL : a.id, b.k ? 0LL : b.id);
}

// The operations that the values `outs` depend on, each counted once.
[[maybe_unused]] static OpTally count_reachable(const Cnt* outs, int n) {
  OpTally t;
  std::vector<char> mark(g_ts.node.size(), 0);
  std::vector<long long> stack;
  for (int i = 0; i < n; ++i)
    if (!outs[i].k) stack.push_back(outs[i].id);
  while (!stack.empty()) {
    const long long id = stack.back();
    stack.pop_back();
    if (id <= 0 || mark[id]) continue;
    mark[id] = 1;
    const int op = std::get<0>(g_ts.node[id]);
    if (op < 0) continue;  // an input
    switch (op) {
      case OP_ADD: case OP_SUB: ++t.add; break;
      case OP_MUL: ++t.mul; break;
      case OP_DIV: ++t.div; break;
      case OP_SQRT: ++t.sqrt; break;
      case OP_EXP: case OP_EXPM1: ++t.exp; break;
      case OP_ERF: ++t.erf; break;
      case OP_POW: ++t.pow; break;
      default: break;  // negation, absolute value: free
    }
    stack.push_back(std::get<1>(g_ts.node[id]));
    stack.push_back(std::get<2>(g_ts.node[id]));
  }
  return t;
}

// The formulas are __host__ __device__; the tally runs on the host only (the
// device pass of this file compiles the counting type but never runs it).
#ifdef __CUDA_ARCH__
#define HGKS_RECORD(op, a, b, r)
#else
#define HGKS_RECORD(op, a, b, r) record(op, a, b, r)
#endif
#define CNT_FN __host__ __device__ inline

CNT_FN bool is_exactly(const Cnt& a, double x) { return a.k && a.v == x; }

CNT_FN Cnt var_result(double v) {
  Cnt c;
  c.v = v;
  c.k = false;
  return c;
}

// A binary operation: folded when both operands are constants, else
// recorded (or passed through for the free identities).
CNT_FN Cnt binary(int op, const Cnt& a, const Cnt& b, double v) {
  if (a.k && b.k) return Cnt(v);
  Cnt r = var_result(v);
  HGKS_RECORD(op, a, b, r);
  return r;
}

CNT_FN Cnt operator+(Cnt a, Cnt b) {
  if (is_exactly(a, 0.0)) return b;
  if (is_exactly(b, 0.0)) return a;
  return binary(OP_ADD, a, b, a.v + b.v);
}
CNT_FN Cnt operator-(Cnt a) {
  if (a.k) return Cnt(-a.v);
  Cnt r = var_result(-a.v);
  HGKS_RECORD(OP_NEG, a, Cnt(0.0), r);
  return r;
}
CNT_FN Cnt operator-(Cnt a, Cnt b) {
  if (is_exactly(b, 0.0)) return a;
  if (is_exactly(a, 0.0)) return -b;
  return binary(OP_SUB, a, b, a.v - b.v);
}
CNT_FN Cnt operator*(Cnt a, Cnt b) {
  if (is_exactly(a, 0.0) || is_exactly(b, 0.0)) return Cnt(0.0);
  if (is_exactly(a, 1.0)) return b;
  if (is_exactly(b, 1.0)) return a;
  if (is_exactly(a, -1.0)) return -b;
  if (is_exactly(b, -1.0)) return -a;
  return binary(OP_MUL, a, b, a.v * b.v);
}
CNT_FN Cnt operator/(Cnt a, Cnt b) {
  if (is_exactly(b, 1.0) || is_exactly(a, 0.0)) return a;
  return binary(OP_DIV, a, b, a.v / b.v);
}
CNT_FN Cnt& operator+=(Cnt& a, Cnt b) { return a = a + b; }
CNT_FN Cnt& operator-=(Cnt& a, Cnt b) { return a = a - b; }
CNT_FN Cnt& operator*=(Cnt& a, Cnt b) { return a = a * b; }
CNT_FN bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
CNT_FN bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
CNT_FN bool operator<=(Cnt a, Cnt b) { return a.v <= b.v; }
CNT_FN bool operator>=(Cnt a, Cnt b) { return a.v >= b.v; }
CNT_FN bool operator==(Cnt a, Cnt b) { return a.v == b.v; }
CNT_FN bool operator!=(Cnt a, Cnt b) { return a.v != b.v; }

CNT_FN Cnt unary(int op, const Cnt& x, double v) {
  if (x.k) return Cnt(v);
  Cnt r = var_result(v);
  HGKS_RECORD(op, x, Cnt(0.0), r);
  return r;
}

// Overloads found by argument-dependent lookup in the templated formulas.
CNT_FN Cnt tsqrt(Cnt x) { return unary(OP_SQRT, x, ::sqrt(x.v)); }
CNT_FN Cnt texp(Cnt x) { return unary(OP_EXP, x, ::exp(x.v)); }
CNT_FN Cnt texpm1(Cnt x) { return unary(OP_EXPM1, x, ::expm1(x.v)); }
CNT_FN Cnt terf(Cnt x) { return unary(OP_ERF, x, ::erf(x.v)); }
CNT_FN Cnt tpow(Cnt x, Cnt y) { return binary(OP_POW, x, y, ::pow(x.v, y.v)); }
CNT_FN Cnt tabs(Cnt x) { return unary(OP_ABS, x, ::fabs(x.v)); }

// A fresh per-face value (an input with its own value number).
inline Cnt fresh(double v) {
  Cnt c = var_result(v);
  c.id = g_ts.next++;
  g_ts.node.emplace_back(-1, 0LL, 0LL);
  return c;
}

namespace {

// Gas constants of a configuration, as per-run constants.
Gas<Cnt> count_gas(const hgks_config& c) {
  Gas<Cnt> g;
  g.gamma = Cnt(c.gamma);
  g.gm1 = Cnt(c.gamma - 1.0);
  g.K = Cnt((5.0 - 3.0 * c.gamma) / (c.gamma - 1.0));
  g.pr_fix = Cnt(1.0 / c.prandtl - 1.0);
  g.visc_law = c.visc;
  g.mu_ref = Cnt(c.mu_ref);
  g.T_ref_inv = Cnt(1.0 / c.T_ref);
  g.visc_exp = Cnt(c.visc_exp);
  g.tau_num_C = Cnt(c.flux == HGKS_FLUX_FULL ? c.tau_num_C : 0.0);
  g.rho_r = Cnt(c.rho_ref);
  g.p_r = Cnt(c.p_ref);
  g.h_r = Cnt(c.gamma / (c.gamma - 1.0) * c.p_ref);
  return g;
}

// A per-face value: a smooth sample around the reference state (the values
// only steer the compatibility state's half-space terms, never a branch of
// the count).
Cnt sample(int i, int k, const hgks_config& c) {
  const double base[5] = {0.02, 0.3, -0.2, 0.1, 0.05 * c.p_ref};
  return fresh(base[i] * (1.0 + 0.01 * k));
}


// Tally of the three parts of one face's work in (MODE, FLUX, STAGE):
// out[0..2] = face fields of one point, t1 pass of one point, t2 pass and
// flux of one face (4 Gauss points, weights, the face-flux scaling).
template <int MODE, int FLUX>
void tally_face(const hgks_config& c, int stage, OpTally out[3]) {
  constexpr int NV = SweepLayout<FLUX>::NV;
  constexpr int NFF = SweepLayout<FLUX>::NFF;
  constexpr int NT1 = SweepLayout<FLUX>::NT1;
  const Gas<Cnt> gas = count_gas(c);
  g_ts = TallyState();
  // Phase 1: face fields of one point from its six cells.
  constexpr int NH1 = 1;
  Cnt qa[5][6];
  for (int i = 0; i < 5; ++i)
    for (int k = 0; k < 6; ++k) qa[i][k] = sample(i, k, c);
  Cnt ff1[NFF];
  g_ts.seen.clear();
  face_fields_cells<Cnt, MODE, FLUX, NH1>(qa, fresh(0.1), fresh(0.1), gas, 0, ff1);
  out[0] = count_reachable(ff1, NFF);
  // Phase 2: the t1 pass of one point (five face points along t1).
  constexpr int NH = 5;
  Cnt ff[NFF * NH], tb[NT1 * NH];
  for (int f = 0; f < NFF; ++f)
    for (int h = 0; h < NH; ++h) ff[f * NH + h] = fresh(ff1[f].v * (1.0 + 0.01 * h));
  g_ts.seen.clear();
  for (int grp = 0; grp < 2 * NV / 5; ++grp) t1_pass_group<Cnt, MODE, NV, NH>(ff, tb, 2, 1, grp);
  Cnt t1out[NT1];
  for (int f = 0; f < NT1; ++f) t1out[f] = tb[f * NH + 2];
  out[1] = count_reachable(t1out, NT1);
  for (int f = 0; f < NT1; ++f)
    for (int h = 0; h < NH; ++h) tb[f * NH + h] = fresh(tb[f * NH + 2].v * (1.0 + 0.01 * h));
  // Phase 3: per t1 abscissa, the t2 pass of every field (values and
  // t2-derivatives of the states, values of their t1-derivatives and normal
  // slopes), the widths' scaling of the tangential derivatives, the flux at
  // both t2 abscissae, the Gauss sum and the face-flux scaling.
  const Cnt rh1 = fresh(10.0), rh2 = fresh(10.0), dt = Cnt(1e-3);
  constexpr int NS = FLUX == FLUX_FULL ? 3 : 1;
  g_ts.seen.clear();
  Cnt Fs[10];
  for (int m1 = 0; m1 < 2; ++m1) {
    PointState<Cnt> st[2][NS];
    for (int s = 0; s < NS; ++s)
      for (int i = 0; i < 5; ++i) {
        const int k = 5 * s + i;
        const Cnt* sv = tb + (4 * k + m1) * NH + 2;
        const Cnt* sdv = tb + (4 * k + 2 + m1) * NH + 2;
        const Cnt* ss = tb + (4 * NV + 2 * k + m1) * NH + 2;
        Cnt v[2], dd[2], vd[2], vs[2];
        tangential<MODE>(sv[-2], sv[-1], sv[0], sv[1], sv[2], v, dd);
        tangential_val<MODE>(sdv[-2], sdv[-1], sdv[0], sdv[1], sdv[2], vd);
        tangential_val<MODE>(ss[-2], ss[-1], ss[0], ss[1], ss[2], vs);
        for (int m2 = 0; m2 < 2; ++m2) {
          st[m2][s].q[i] = v[m2];
          st[m2][s].dq[0][i] = vs[m2];
          st[m2][s].dq[1][i] = vd[m2] * rh1;
          st[m2][s].dq[2][i] = dd[m2] * rh2;
        }
      }
    for (int m2 = 0; m2 < 2; ++m2) {
      Cnt F[5], dF[5];
      if constexpr (FLUX == FLUX_SMOOTH) flux_smooth(st[m2][0], gas, stage == 1, F, dF);
      else flux_full(st[m2][0], st[m2][1], st[m2][2], gas, dt, F, dF);
      for (int i = 0; i < 5; ++i) {
        if (stage == 1) Fs[i] += F[i];
        Fs[5 + i] += dF[i];
      }
    }
  }
  for (int i = 0; i < 10; ++i)
    if (stage == 1 || i >= 5) Fs[i] = Cnt(0.25) * Fs[i];
  // The second stage stores dF only (Eq. (6)).
  out[2] = stage == 1 ? count_reachable(Fs, 10) : count_reachable(Fs + 5, 5);
}

void store(const OpTally& t, double* o) {
  o[0] = double(t.add);
  o[1] = double(t.mul);
  o[2] = double(t.div);
  o[3] = double(t.sqrt);
  o[4] = double(t.exp);
  o[5] = double(t.erf);
  o[6] = double(t.pow);
}

}  // namespace
}  // namespace hgks

extern "C" hgks_status hgks_count_flops(const hgks_config* cfg, int stage, double* out) {
  if (!cfg || !out || (stage != 1 && stage != 2)) return HGKS_E_INVAL;
  if (!hgks::validate_config(*cfg).empty()) return HGKS_E_INVAL;
  if (cfg->recon_vars == 1 && cfg->recon != HGKS_RECON_LINEAR) return HGKS_E_UNSUPPORTED;
  hgks::OpTally t[3];
  const int m = cfg->recon, f = cfg->flux;
#define HGKS_FACE(M, F) \
  if (m == M && f == F) hgks::tally_face<M, F>(*cfg, stage, t);
  HGKS_FACE(0, 0) HGKS_FACE(1, 0) HGKS_FACE(2, 0) HGKS_FACE(0, 1) HGKS_FACE(1, 1) HGKS_FACE(2, 1)
#undef HGKS_FACE
  for (int p = 0; p < 3; ++p) hgks::store(t[p], out + 7 * p);
  return HGKS_OK;
}
