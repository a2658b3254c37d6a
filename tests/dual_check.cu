// Host-side check of the dual-number arithmetic used by the derivative-carrying
// step: prints, for each case, the value and derivative parts of f(x + e) at a
// point (the test compares them with closed forms and central differences).
#include <cstdio>

#include "../paper_2111_04577_gb300/csrc/dual.cuh"

using pf::Dual;

template <class F>
static void show(const char* name, F f, double x) {
  const Dual y = f(Dual(x, 1.0));
  std::printf("%s %.17g %.17g %.17g\n", name, x, y.v, y.d);
}

int main() {
  const double xs[] = {0.3, 1.7, 4.0};
  for (double x : xs) {
    show("sqrt", [](Dual a) { return sqrt(a); }, x);
    show("rsqrt", [](Dual a) { return rsqrt(a); }, x);
    show("exp", [](Dual a) { return exp(a); }, x);
    show("expm1", [](Dual a) { return expm1(a); }, x);
    show("exp2", [](Dual a) { return exp2(a); }, x);
    show("log2", [](Dual a) { return log2(a); }, x);
    show("neg", [](Dual a) { return fabs(-a); }, x);
    show("quot", [](Dual a) { return (a * a + 1.0) / (2.0 - a * 0.25); }, x);
    show("chain", [](Dual a) {  // a composite like the step's: compound assignment, division, functions
      Dual s = a;
      s *= exp(-a);
      s /= (1.0 + a * a);
      s += sqrt(a) * log2(1.0 + a);
      s -= expm1(-0.5 * a) / a;
      return s;
    }, x);
  }
  return 0;
}
