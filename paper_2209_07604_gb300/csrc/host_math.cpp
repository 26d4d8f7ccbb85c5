// Host-side numerical set-up of libfhs (FP64): Daubechies filters by spectral
// factorisation, the Kaiser-Bessel kernel and its Fourier transform, and the
// w-projection kernels of each w-plane (Sec. 3.2).  Written independently of
// any test oracle; the tests compare the two.
#include "fhs_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace fhs {

using cd = std::complex<double>;

// Modified Bessel function I0 by its power series sum_k ((x/2)^2)^k / (k!)^2.
double bessel_i0(double x) {
    const double q = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 500; ++k) {
        term *= q / (double(k) * double(k));
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

double kb_beta(int J, double os) {
    const double a = double(J) / os;
    return M_PI * std::sqrt(a * a * (os - 0.5) * (os - 0.5) - 0.8);
}

// Continuous Fourier transform of phi(t) = I0(beta sqrt(1-(2t/J)^2))/I0(beta):
// J sinh(z)/z / I0(beta) with z^2 = beta^2 - (pi J nu)^2 (sin form for z^2 < 0).
double kb_hat(double nu, int J, double beta) {
    const double z2 = beta * beta - (M_PI * J * nu) * (M_PI * J * nu);
    double r;
    if (z2 > 0) {
        const double z = std::sqrt(z2);
        r = std::sinh(z) / z;
    } else if (z2 < 0) {
        const double z = std::sqrt(-z2);
        r = std::sin(z) / z;
    } else {
        r = 1.0;
    }
    return J * r / bessel_i0(beta);
}

// Roots of a real polynomial (coefficients in descending powers) by the
// Durand-Kerner (Weierstrass) simultaneous iteration, then Newton polishing.
static std::vector<cd> poly_roots(const std::vector<double> &desc) {
    const int n = int(desc.size()) - 1;
    std::vector<cd> r(n);
    if (n <= 0) return r;
    std::vector<cd> a(n + 1);
    for (int i = 0; i <= n; ++i) a[i] = desc[i] / desc[0];   // monic
    auto eval = [&](cd z) {
        cd v = a[0];
        for (int i = 1; i <= n; ++i) v = v * z + a[i];
        return v;
    };
    auto deriv = [&](cd z) {
        cd v = double(n) * a[0];
        for (int i = 1; i < n; ++i) v = v * z + double(n - i) * a[i];
        return v;
    };
    const cd seed(0.4, 0.9);
    for (int i = 0; i < n; ++i) r[i] = std::pow(seed, i);
    for (int it = 0; it < 2000; ++it) {
        double delta = 0.0;
        for (int i = 0; i < n; ++i) {
            cd den = 1.0;
            for (int j = 0; j < n; ++j)
                if (j != i) den *= (r[i] - r[j]);
            const cd step = eval(r[i]) / den;
            r[i] -= step;
            delta = std::max(delta, std::abs(step));
        }
        if (delta < 1e-15) break;
    }
    for (int i = 0; i < n; ++i)
        for (int it = 0; it < 5; ++it) {
            const cd d = deriv(r[i]);
            if (std::abs(d) == 0.0) break;
            r[i] -= eval(r[i]) / d;
        }
    return r;
}

// db_p low-pass filter (2p taps).  |m0(w)|^2 = cos^{2p}(w/2) P(sin^2(w/2)),
// P(y) = sum_{k<p} C(p-1+k,k) y^k.  Each root y_k of P yields the zero pair
// z + 1/z = 2 - 4 y_k of H(z) = sum h[n] z^-n; the one inside the unit circle
// is kept (minimum phase), the remaining p zeros sit at z = -1.
std::vector<double> daubechies(int p) {
    std::vector<double> ydesc(p);       // descending powers of y
    for (int k = 0; k < p; ++k) {
        double c = 1.0;                 // C(p-1+k, k)
        for (int i = 1; i <= k; ++i) c = c * double(p - 1 + i) / double(i);
        ydesc[p - 1 - k] = c;
    }
    std::vector<cd> zeros;
    if (p > 1) {
        for (const cd &yk : poly_roots(ydesc)) {
            const cd b = 2.0 - 4.0 * yk;
            const cd disc = std::sqrt(b * b - 4.0);
            const cd z1 = 0.5 * (b + disc), z2 = 0.5 * (b - disc);
            zeros.push_back(std::abs(z1) < 1.0 ? z1 : z2);
        }
    }
    std::vector<cd> poly{1.0};
    auto mul = [&](cd root) {          // poly *= (1 - root z^-1), ascending powers of z^-1
        std::vector<cd> out(poly.size() + 1, 0.0);
        for (size_t i = 0; i < poly.size(); ++i) {
            out[i] += poly[i];
            out[i + 1] -= root * poly[i];
        }
        poly.swap(out);
    };
    for (int i = 0; i < p; ++i) mul(-1.0);
    for (const cd &z : zeros) mul(z);
    std::vector<double> h(poly.size());
    double s = 0.0;
    for (size_t i = 0; i < poly.size(); ++i) {
        h[i] = poly[i].real();
        s += h[i];
    }
    for (double &v : h) v *= std::sqrt(2.0) / s;
    return h;
}

// Phase profile of the w-term chirp over the K-point grid: n^2 on the image
// support |n| <= N/2, then a slope falling linearly from N to 0 at |n| = K/2
// so the periodic extension is smooth (the image is zero there, so any
// extension leaves the untruncated row unchanged).
double chirp_phase(double n_abs, int N, int K) {
    const double hN = 0.5 * N, hK = 0.5 * K;
    if (n_abs <= hN) return n_abs * n_abs;
    return hN * hN + double(N) / (hK - hN) * (hK * (n_abs - hN) - 0.5 * (n_abs * n_abs - hN * hN));
}

// Truncated, unit-sum w-kernel of plane value wp along one axis:
// chat(j) = (1/K) sum_n exp(i pi wp dl^2 psi(n)) exp(-2 pi i j n / K), j = -h..h.
void wkernel(double wp, int N, int K, double pixel_size, int h, cd *out) {
    const int S = 2 * h + 1;
    if (h == 0) {
        out[0] = 1.0;
        return;
    }
    const double a = wp * pixel_size * pixel_size;
    std::vector<cd> chirp(K);
    for (int i = 0; i < K; ++i) {
        const double n = double(i - K / 2);
        chirp[i] = std::polar(1.0, M_PI * a * chirp_phase(std::fabs(n), N, K));
    }
    cd total = 0.0;
    for (int s = 0; s < S; ++s) {
        const int j = s - h;
        cd acc = 0.0;
        for (int i = 0; i < K; ++i) {
            const double n = double(i - K / 2);
            acc += chirp[i] * std::polar(1.0, -2.0 * M_PI * double(j) * n / double(K));
        }
        out[s] = acc / double(K);
        total += out[s];
    }
    for (int s = 0; s < S; ++s) out[s] /= total;
}

}  // namespace fhs
