// Bin enthalpies from the Debye heat capacity: the helper a caller uses to turn a grain's
// temperature grid into the enthalpy bins E_i = H(T_i) that heat_set_grains takes (Sec. 2:
// the bins sit on a user-supplied temperature grid; the enthalpy is the integral of the
// grain's heat capacity).  Host code only.
#include <cmath>

#include "../../include/heat.h"

namespace {

constexpr double kBoltzmann = 1.380649e-16;  // erg/K (CODATA 2018, exact)

// D(y) = int_0^y x^3 / (e^x - 1) dx.
//   y < 1: x^3/(e^x - 1) = x^2 * (x/(e^x - 1)) and x/(e^x - 1) = sum_n B_n x^n / n!
//          (Bernoulli numbers, B_1 = -1/2), integrated term by term:
//          D = y^3/3 - y^4/8 + sum_{k>=1} B_2k y^(2k+3) / ((2k+3) (2k)!); the series
//          converges for y < 2 pi, and at y < 1 its terms fall by (y / 2 pi)^2 < 0.026 each.
//   y >= 1: D = pi^4/15 - sum_{m>=1} e^{-m y} (y^3/m + 3 y^2/m^2 + 6 y/m^3 + 6/m^4), from
//          expanding 1/(e^x - 1) = sum_m e^{-m x} and integrating x^3 e^{-m x} from y to
//          infinity; terms past e^{-m y} < 1e-18 are dropped.
double bose3(double y) {
    if (!(y > 0.0)) return 0.0;
    if (y < 1.0) {
        // B_2k, k = 1..12
        static const double B[12] = {1.0 / 6.0,           -1.0 / 30.0,        1.0 / 42.0,
                                     -1.0 / 30.0,         5.0 / 66.0,         -691.0 / 2730.0,
                                     7.0 / 6.0,           -3617.0 / 510.0,    43867.0 / 798.0,
                                     -174611.0 / 330.0,   854513.0 / 138.0,   -236364091.0 / 2730.0};
        const double y2 = y * y;
        double s = 0.0;
        double pw = y2 * y2 * y;  // y^(2k+3) at k = 1
        double fact = 2.0;        // (2k)! at k = 1
        for (int k = 1; k <= 12; ++k) {
            s += B[k - 1] * pw / ((2.0 * k + 3.0) * fact);
            pw *= y2;
            fact *= (2.0 * k + 1.0) * (2.0 * k + 2.0);
        }
        return y2 * y / 3.0 - y2 * y2 / 8.0 + s;
    }
    const double pi4_15 = M_PI * M_PI * M_PI * M_PI / 15.0;
    double tail = 0.0;
    const int mmax = (int)std::ceil(41.5 / y) + 1;  // e^{-m y} < 1e-18 beyond
    for (int m = mmax; m >= 1; --m) {               // smallest terms first
        const double em = std::exp(-m * y);
        if (em == 0.0) continue;
        const double mi = 1.0 / m;
        tail += em * mi * (y * y * y + mi * (3.0 * y * y + mi * (6.0 * y + mi * 6.0)));
    }
    return pi4_15 - tail;
}

}  // namespace

extern "C" double heat_debye_enthalpy(double theta_D, double n_atoms, double T) {
    if (!(theta_D > 0.0) || !(n_atoms > 0.0) || !(T >= 0.0) || !std::isfinite(theta_D) || !std::isfinite(n_atoms) ||
        !std::isfinite(T))
        return NAN;
    if (T == 0.0) return 0.0;
    // H(T) = 9 N k T (T / theta)^3 D(theta / T): the internal energy of 3N Debye modes above
    // the zero-point energy
    const double r = T / theta_D;
    return 9.0 * n_atoms * kBoltzmann * T * r * r * r * bose3(theta_D / T);
}
