// Host check of the packed-pair reconstructions and their transposes
// (csrc/packed.cuh, csrc/adjoint.cuh) against the scalar functions they
// restate (csrc/recon.cuh, csrc/adjoint.cuh), in FP32 on seeded stencils:
// each half of a packed evaluation must give the scalar result of its
// stencil to FP32 rounding.  On the host a pair operation is the two scalar
// operations it stands for, so this checks the packed algebra (every term,
// sign and index of the restatement), not the device's rounding.  Also a
// constant stencil, where WENO-Z's smoothness indicators vanish.  Prints
// the largest scaled difference of the reconstructions and of the
// transposes (whose 1/beta^2 and 1/(eps + beta)^3 factors amplify FP32
// rounding: the scalar FP32 transpose itself is ~3e-5 from its FP64
// evaluation on these stencils, the packed one no further).
// Test support: built and run by tests/test_packed_pairs.py; not part of the
// library.
#include <cmath>
#include <cstdio>
#include <random>

#include "adjoint.cuh"

using namespace hgks;

namespace {

double worst[2] = {0.0, 0.0};  // forward reconstructions, transposes
int part = 0;

void record(float a, float b, float scale) {
  const double e = std::fabs(double(a) - double(b)) / (scale > 0 ? scale : 1.0);
  if (e > worst[part]) worst[part] = e;
  if (!std::isfinite(a)) worst[part] = 1e30;
}

template <int MODE>
void check(const float qa[5], const float qb[5], std::mt19937_64& rng) {
  std::uniform_real_distribution<float> u(-1.f, 1.f);
  float scale = 0.f;
  for (int k = 0; k < 5; ++k) scale = std::fmax(scale, std::fmax(std::fabs(qa[k]), std::fabs(qb[k])));
  float2 q2[5];
  for (int k = 0; k < 5; ++k) q2[k] = make_float2(qa[k], qb[k]);
  part = 0;
  // WENO5 end values
  if (MODE != RECON_LINEAR) {
    float2 L2, R2;
    weno5_pair_x2<MODE>(q2[0], q2[1], q2[2], q2[3], q2[4], L2, R2);
    float La, Ra, Lb, Rb;
    weno5_pair<MODE>(qa[0], qa[1], qa[2], qa[3], qa[4], La, Ra);
    weno5_pair<MODE>(qb[0], qb[1], qb[2], qb[3], qb[4], Lb, Rb);
    record(L2.x, La, scale);
    record(R2.x, Ra, scale);
    record(L2.y, Lb, scale);
    record(R2.y, Rb, scale);
  }
  // tangential values and derivatives
  {
    float2 v2[2], d2[2];
    if constexpr (MODE == RECON_LINEAR) tangential_linear_x2(q2[0], q2[1], q2[2], q2[3], q2[4], v2, d2);
    else tangential_weno_x2<MODE>(q2[0], q2[1], q2[2], q2[3], q2[4], v2, d2);
    float va[2], da[2], vb[2], db[2];
    tangential<MODE>(qa[0], qa[1], qa[2], qa[3], qa[4], va, da);
    tangential<MODE>(qb[0], qb[1], qb[2], qb[3], qb[4], vb, db);
    for (int m = 0; m < 2; ++m) {
      record(v2[m].x, va[m], scale);
      record(v2[m].y, vb[m], scale);
      record(d2[m].x, da[m], scale);
      record(d2[m].y, db[m], scale);
    }
  }
  if (MODE == RECON_LINEAR) return;
  part = 1;
  // transposes, with random cotangents
  {
    const float gLa = u(rng), gRa = u(rng), gLb = u(rng), gRb = u(rng);
    float2 c2[5];
    float ca[5] = {0, 0, 0, 0, 0}, cb[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 5; ++k) c2[k] = make_float2(0.f, 0.f);
    weno5_pair_vjp_x2<MODE>(q2, make_float2(gLa, gLb), make_float2(gRa, gRb), c2);
    weno5_pair_vjp<MODE>(qa, gLa, gRa, ca);
    weno5_pair_vjp<MODE>(qb, gLb, gRb, cb);
    float sa = 0.f, sb = 0.f;
    for (int k = 0; k < 5; ++k) {
      sa = std::fmax(sa, std::fabs(ca[k]));
      sb = std::fmax(sb, std::fabs(cb[k]));
    }
    for (int k = 0; k < 5; ++k) {
      record(c2[k].x, ca[k], sa + 1.f);
      record(c2[k].y, cb[k], sb + 1.f);
    }
  }
  {
    const float gva[2] = {u(rng), u(rng)}, gda[2] = {u(rng), u(rng)};
    const float gvb[2] = {u(rng), u(rng)}, gdb[2] = {u(rng), u(rng)};
    const float2 gv2[2] = {make_float2(gva[0], gvb[0]), make_float2(gva[1], gvb[1])};
    const float2 gd2[2] = {make_float2(gda[0], gdb[0]), make_float2(gda[1], gdb[1])};
    float2 c2[5];
    float ca[5] = {0, 0, 0, 0, 0}, cb[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 5; ++k) c2[k] = make_float2(0.f, 0.f);
    tangential_vjp_x2<MODE>(q2, gv2, gd2, c2);
    tangential_vjp<MODE>(qa, gva, gda, ca);
    tangential_vjp<MODE>(qb, gvb, gdb, cb);
    float sa = 0.f, sb = 0.f;
    for (int k = 0; k < 5; ++k) {
      sa = std::fmax(sa, std::fabs(ca[k]));
      sb = std::fmax(sb, std::fabs(cb[k]));
    }
    for (int k = 0; k < 5; ++k) {
      record(c2[k].x, ca[k], sa + 1.f);
      record(c2[k].y, cb[k], sb + 1.f);
    }
  }
}

}  // namespace

int main() {
  std::mt19937_64 rng(2024);
  std::uniform_real_distribution<float> u(-1.f, 1.f);
  for (int trial = 0; trial < 2000; ++trial) {
    // smooth part (a quadratic) plus noise of varying size: weights from near
    // linear to strongly nonlinear
    float qa[5], qb[5];
    const float noise = trial % 4 == 0 ? 1e-3f : (trial % 4 == 1 ? 0.05f : (trial % 4 == 2 ? 0.5f : 2.f));
    const float a0 = u(rng), a1 = u(rng), a2 = 0.2f * u(rng);
    const float b0 = u(rng), b1 = u(rng), b2 = 0.2f * u(rng);
    for (int k = 0; k < 5; ++k) {
      const float x = float(k - 2);
      qa[k] = a0 + a1 * x + a2 * x * x + noise * u(rng);
      qb[k] = b0 + b1 * x + b2 * x * x + noise * u(rng);
    }
    if (trial % 50 == 7)
      for (int k = 0; k < 5; ++k) qa[k] = 0.75f;  // constant: all indicators vanish
    check<RECON_LINEAR>(qa, qb, rng);
    check<RECON_WENO_JS>(qa, qb, rng);
    check<RECON_WENO_Z>(qa, qb, rng);
  }
  std::printf("%.3e %.3e\n", worst[0], worst[1]);
  return 0;
}
