// count_collide_flops.cpp -- flops of the oracle's collide, counted by instrumentation.
//
// TEST INFRASTRUCTURE ONLY (like the rest of oracle/). The oracle's own C source is compiled here
// with `double` replaced by an operation-counting scalar type: every binary +, -, *, / on it adds
// one to a counter (the oracle is built without contraction, so it has no fused multiply-adds;
// sign changes and comparisons are not counted). The program runs the oracle's collide on one
// site and prints the count: the algorithmic floating-point work of one site update in the
// oracle's plain formulation (moments, the Hermite equilibrium written per population, BGK
// relaxation with the gravity shift). Propagate is a copy and does no arithmetic.
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>

struct Flop {
    double v;
    static long long n;
    Flop() : v(0.0) {}
    Flop(double x) : v(x) {}  // NOLINT: implicit, as a drop-in for double
    Flop& operator+=(Flop o) { ++n; v += o.v; return *this; }
    Flop& operator-=(Flop o) { ++n; v -= o.v; return *this; }
    Flop& operator*=(Flop o) { ++n; v *= o.v; return *this; }
    Flop& operator/=(Flop o) { ++n; v /= o.v; return *this; }
    Flop operator-() const { return Flop(-v); }
    explicit operator double() const { return v; }
};
long long Flop::n = 0;
static Flop operator+(Flop a, Flop b) { ++Flop::n; return Flop(a.v + b.v); }
static Flop operator-(Flop a, Flop b) { ++Flop::n; return Flop(a.v - b.v); }
static Flop operator*(Flop a, Flop b) { ++Flop::n; return Flop(a.v * b.v); }
static Flop operator/(Flop a, Flop b) { ++Flop::n; return Flop(a.v / b.v); }
static bool operator>(Flop a, Flop b) { return a.v > b.v; }
static bool operator<(Flop a, Flop b) { return a.v < b.v; }
static Flop sqrt(Flop a) { ++Flop::n; return Flop(std::sqrt(a.v)); }

// the system headers above are already included, so only the oracle's own code sees the macro
#define double Flop
#include "d2q37_oracle.c"
#undef double

int main() {
    setup();
    Flop f[NPOP];
    for (int i = 0; i < NPOP; ++i) f[i] = W[i];  // any state: the count does not depend on values
    f[3] = f[3] * Flop(1.01);
    Flop::n = 0;
    collide_site(f, Flop(0.9), Flop(1e-4), Flop(-2e-4));
    printf("%lld\n", Flop::n);
    return 0;
}
