// breakpoints.cu -- the SAX breakpoints (Sec. 2.2): the N(0,1) quantiles
// beta_j = PhiInv(j / c), j = 1 .. c-1, each the double nearest the real
// quantile (correctly rounded), so that every correct implementation of the
// definition yields the same table bit for bit and a PAA value is assigned
// the same symbol whoever computes it.
//
// Method (host code, double-double arithmetic, ~104-bit significands):
//   Phi(x) = 1/2 + phi(x) * S(x),  S(x) = x + x^3/3 + x^5/(3*5) + ...
//   (the series of Phi in powers of x with all terms of one sign), phi(x) =
//   exp(-x^2/2) / sqrt(2 pi), exp by a Taylor series after halving the
//   argument six times, then squaring six times.
//   A double estimate of the root is refined by two double-double Newton
//   steps, rounded to the nearest double c, and c is certified: the CDF at
//   the two midpoints between c and its neighbours must bracket p, each by a
//   margin far above the evaluation error; otherwise c moves to the neighbour
//   the bracket points at and is certified again.
// Only the lower half (p < 1/2, beta < 0) is computed; the upper half
// follows from the symmetry PhiInv(1 - p) = -PhiInv(p), and beta_{c/2} = 0.
#include <cmath>

#include "messi_internal.cuh"

namespace messi {
namespace {

struct DD {
    double hi, lo;
};

DD quick_two_sum(double a, double b)   // |a| >= |b|
{
    const double s = a + b;
    return {s, b - (s - a)};
}
DD two_sum(double a, double b)
{
    const double s = a + b;
    const double bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
DD two_prod(double a, double b)
{
    const double p = a * b;
    return {p, std::fma(a, b, -p)};
}
DD add(DD a, DD b)
{
    DD s = two_sum(a.hi, b.hi);
    const DD t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
DD neg(DD a) { return {-a.hi, -a.lo}; }
DD sub(DD a, DD b) { return add(a, neg(b)); }
DD mul(DD a, DD b)
{
    DD p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}
DD mul_d(DD a, double b)
{
    DD p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return quick_two_sum(p.hi, p.lo);
}
DD div(DD a, DD b)
{
    const double q1 = a.hi / b.hi;
    DD r = sub(a, mul_d(b, q1));
    const double q2 = r.hi / b.hi;
    r = sub(r, mul_d(b, q2));
    const double q3 = r.hi / b.hi;
    DD q = quick_two_sum(q1, q2);
    return add(q, DD{q3, 0.0});
}
DD sqrt_dd(DD a)
{
    const double s = std::sqrt(a.hi);
    // one Newton step from the double root: s + (a - s^2) / (2 s)
    const DD r = sub(a, two_prod(s, s));
    return add(DD{s, 0.0}, DD{r.hi / (2.0 * s), 0.0});
}

// pi as a double-double (the double nearest pi, and the double nearest the rest)
constexpr DD kPi = {3.141592653589793116, 1.2246467991473532e-16};

DD inv_sqrt_2pi()
{
    const DD two_pi = {2.0 * kPi.hi, 2.0 * kPi.lo};
    return div(DD{1.0, 0.0}, sqrt_dd(two_pi));
}

// exp(y) for -8 <= y <= 0
DD exp_dd(DD y)
{
    const int halvings = 6;
    const DD z = {std::ldexp(y.hi, -halvings), std::ldexp(y.lo, -halvings)};   // exact
    DD sum = {1.0, 0.0}, term = {1.0, 0.0};
    for (int n = 1; n < 40; ++n) {
        term = div(mul(term, z), DD{(double)n, 0.0});
        sum = add(sum, term);
        if (std::fabs(term.hi) < 1e-36) break;
    }
    for (int i = 0; i < halvings; ++i) sum = mul(sum, sum);
    return sum;
}

// Phi(x) for -9 <= x <= 0: 1/2 + phi(x) (x + x^3/3 + x^5/15 + ...)
DD cdf_dd(DD x)
{
    const DD x2 = mul(x, x);
    DD term = x, s = x;
    for (int n = 1; n < 400; ++n) {
        term = div(mul(term, x2), DD{(double)(2 * n + 1), 0.0});
        s = add(s, term);
        if (std::fabs(term.hi) < 1e-40 * std::fabs(s.hi)) break;
    }
    const DD phi = mul(exp_dd(mul_d(x2, -0.5)), inv_sqrt_2pi());
    return add(DD{0.5, 0.0}, mul(phi, s));
}

DD density_dd(DD x)
{
    return mul(exp_dd(mul_d(mul(x, x), -0.5)), inv_sqrt_2pi());
}

// The double nearest PhiInv(p), 0 < p < 1/2 (p exact in double).
double quantile_rn(double p)
{
    // double estimate: Newton on erfc, kept inside (lo, 0) by bisection when
    // a step leaves it; then double-double Newton steps until they stall
    const double inv_sqrt_2pi_d = 0.3989422804014327;
    double lo = -40.0, hi = 0.0, x = -1.0;
    for (int it = 0; it < 200; ++it) {
        const double f = 0.5 * std::erfc(-x / std::sqrt(2.0)) - p;
        if (f < 0.0) lo = x; else hi = x;
        double nx = x - f / (inv_sqrt_2pi_d * std::exp(-0.5 * x * x));
        if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
        if (nx == x) break;
        x = nx;
    }
    DD r = {x, 0.0};
    for (int it = 0; it < 6; ++it) {
        const DD step = div(sub(cdf_dd(r), DD{p, 0.0}), density_dd(r));
        r = sub(r, step);
        if (std::fabs(step.hi) < 1e-31 * std::fabs(r.hi)) break;
    }
    double c = r.hi + r.lo;
    // certify: Phi(c - gap_below/2) < p < Phi(c + gap_above/2); the CDF is
    // evaluated to ~2^-95 relative, far below the gap at a midpoint unless
    // the quantile lies within ~2^-40 ulp of one (then c stays as it is)
    for (int it = 0; it < 8; ++it) {
        const double below = std::nextafter(c, -INFINITY), above = std::nextafter(c, INFINITY);
        const DD m_lo = quick_two_sum(c, -(c - below) * 0.5), m_hi = quick_two_sum(c, (above - c) * 0.5);
        if (sub(cdf_dd(m_lo), DD{p, 0.0}).hi >= 0.0) { c = below; continue; }   // quantile below m_lo
        if (sub(cdf_dd(m_hi), DD{p, 0.0}).hi <= 0.0) { c = above; continue; }   // quantile above m_hi
        break;
    }
    return c;
}

}  // namespace

void compute_breakpoints(int card, double *beta)
{
    for (int j = 1; 2 * j < card; ++j) beta[j - 1] = quantile_rn((double)j / card);
    for (int j = 1; j < card; ++j) {
        if (2 * j == card) beta[j - 1] = 0.0;
        else if (2 * j > card) beta[j - 1] = -beta[card - j - 1];
    }
}

}  // namespace messi
