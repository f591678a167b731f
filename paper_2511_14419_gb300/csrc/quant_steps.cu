// 9/7 quantisation step table (host).
//
// Paper: §Implementation details (JPEG2000 encoding of the raw image; the
// irreversible path quantises).  The paper gives no step sizes; the
// library uses, for subband b, delta_base / sqrt(G_b) with G_b the squared
// L2 norm of b's 2-D synthesis basis function (the usual energy weighting,
// so equal steps cost equal reconstruction error), written in the JPEG2000
// form 2^(R_b - eps) * (1 + mu / 2^11), R_b = B + gain_b (gain 0 LL, 1 HL
// and LH, 2 HH), eps in 5 bits, mu in 11 bits rounded to nearest.
//
// The 2-D basis of a separable transform is the outer product of 1-D bases,
// so G_b is a product of two 1-D norms.  Each 1-D norm is measured here by
// synthesising a unit impulse through `levels` levels of the 1-D inverse
// 9/7 lifting (whole-sample symmetric extension) on a signal long enough
// that the basis function never reaches the border.
#include <cmath>
#include <vector>

#include "kernels.h"

namespace flowroi {

namespace {

constexpr double kA = -1.586134342059924, kB = -0.052980118572961, kG = 0.882911075530934, kD = 0.443506852043971,
                 kK = 1.230174104914001;

int wsym(int i, int n)
{
    const int period = 2 * (n - 1);
    i %= period;
    if (i < 0) i += period;
    return i <= n - 1 ? i : period - i;
}

// One level of 1-D inverse 9/7 on x[0..n): input is (low band, high band)
// concatenated, output the interleaved signal.
void inverse_level(std::vector<double> &x, int n)
{
    const int nl = (n + 1) / 2;
    std::vector<double> y(n);
    for (int i = 0; i < n; i++) y[i] = (i & 1) ? x[nl + i / 2] / kK : x[i / 2] * kK;
    const double c[4] = {kA, kB, kG, kD};
    for (int s = 3; s >= 0; s--) {
        const int start = (s % 2 == 0) ? 1 : 0;
        for (int i = start; i < n; i += 2) y[i] -= c[s] * (y[wsym(i - 1, n)] + y[wsym(i + 1, n)]);
    }
    for (int i = 0; i < n; i++) x[i] = y[i];
}

// Squared norm of the 1-D synthesis basis of the band `high` at `level`.
double basis_norm(int level, bool high)
{
    const int n = 1 << (level + 6);
    std::vector<double> x(n, 0.0);
    const int band = n >> level;          // length of each band at this level
    const int pos = (high ? band : 0) + band / 2;
    x[pos] = 1.0;
    for (int l = level; l >= 1; l--) inverse_level(x, n >> (l - 1));
    double s = 0.0;
    for (double v : x) s += v * v;
    return s;
}

}  // namespace

int quant_steps(int levels, int bit_depth, double delta_base, float *delta, int *eps, int *mu, double *gain)
{
    if (levels < 1 || levels > kMaxLevels || bit_depth < 1 || bit_depth > 16 || !(delta_base > 0)) return -1;
    int rc = 0;
    std::vector<double> nl(levels + 1), nh(levels + 1);
    for (int l = 1; l <= levels; l++) {
        nl[l] = basis_norm(l, false);
        nh[l] = basis_norm(l, true);
    }
    for (int b = 0; b <= 3 * levels; b++) {
        int l, o;
        if (b == 3 * levels) { l = levels; o = 3; }
        else { l = b / 3 + 1; o = b % 3; }
        double g;
        switch (o) {
        case 0: g = nh[l] * nl[l]; break;  // HL: high horizontally, low vertically
        case 1: g = nl[l] * nh[l]; break;  // LH
        case 2: g = nh[l] * nh[l]; break;  // HH
        default: g = nl[l] * nl[l]; break; // LL
        }
        const double target = delta_base / std::sqrt(g);
        const int gainb = o == 3 ? 0 : (o == 2 ? 2 : 1);
        const int Rb = bit_depth + gainb;
        int e = (int)std::floor(std::log2(target));
        const double m = target / std::ldexp(1.0, e) - 1.0;
        int mi = (int)std::floor(m * 2048.0 + 0.5);
        if (mi == 2048) { mi = 0; e += 1; }
        const int ep = Rb - e;
        if (ep < 0 || ep > 31) rc = -1;
        if (delta) delta[b] = (float)(std::ldexp(1.0, Rb - ep) * (1.0 + mi / 2048.0));
        if (eps) eps[b] = ep;
        if (mu) mu[b] = mi;
        if (gain) gain[b] = g;
    }
    return rc;
}

}  // namespace flowroi
