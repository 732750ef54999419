// Chebyshev coefficients of polynomial operators applied with the
// Chebyshev propagation of the library (mpk_cheb_real): an approximate
// inverse, used as a polynomial preconditioner or a fixed-degree solve.
// Host code only.
#include <cmath>

#include "mpk.h"

extern "C" int mpk_cheb_coeffs_inverse(int32_t M, double c, double r, double *coef) {
    if (M < 0 || !coef || !(r >= 0.0) || !(c > r)) return MPK_ERR_INVALID;
    // 1 / (c + r t) on [-1, 1] equals (1 / s) sum_k (2 - delta_k0) (-q)^k T_k(t)
    // with s = sqrt(c^2 - r^2) and q = (c - s) / r = r / (c + s), the root
    // below 1 of q^2 - (2c/r) q + 1 = 0: the Chebyshev generating function
    // sum_k z^k T_k(t) = (1 - z t) / (1 - 2 z t + z^2) at z = -q.
    const double s = std::sqrt((c - r) * (c + r));
    const double q = r / (c + s);   // the same root, without cancellation for small r
    double qk = 1.0;
    for (int32_t k = 0; k <= M; k++) {
        coef[k] = (k == 0 ? 1.0 : 2.0) * qk / s;
        qk *= -q;
    }
    return MPK_OK;
}
