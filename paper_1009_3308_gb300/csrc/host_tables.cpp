// Host FP64 precompute of the quadrature nodes and Legendre tables.
//
// * Gauss-Legendre nodes/weights of the Gauss-rectangle rule Q_M (Sec. 3,
//   Eq. (quadrule)): Newton's method in the colatitude theta on
//   P_n(cos theta), with the Bonnet recurrence rewritten in y = 1 - cos theta
//   so that nodes near the poles keep full relative accuracy in theta and
//   sin(theta).
// * Orthonormal associated Legendre functions Pt_K^m (the theta part of the
//   scalar harmonics Y_{K,m} of Eq. (sph_har), Condon-Shortley phase
//   included), by the standard orthonormal three-term recurrence in K.  The
//   values are carried as mantissa * 2^e with an integer exponent so that
//   sin(theta)^m never underflows mid-recurrence; values below the binary64
//   range round to zero/subnormal when converted.
#include <cmath>
#include <thread>
#include <vector>

#include "internal.h"

namespace sph {

namespace {
// P_n and D_n = P_n - P_{n-1} at x = 1 - y:
//   (k+1) D_{k+1} = k D_k - (2k+1) y P_k,  P_{k+1} = P_k + D_{k+1}.
void legendre_y(int n, double y, double* P, double* D) {
    double p = 1.0 - y, d = -y;
    for (int k = 1; k < n; ++k) {
        d = (k * d - (2.0 * k + 1.0) * y * p) / (k + 1.0);
        p += d;
    }
    *P = p;
    *D = d;
}
}  // namespace

void gauss_legendre(int n, double* theta, double* x, double* s, double* w) {
    const int nh = (n + 1) / 2;
    for (int i = 0; i < nh; ++i) {
        double th = M_PI * (i + 0.75) / (n + 0.5);
        const bool equator = (n % 2 == 1) && (i == nh - 1);
        if (equator) th = 0.5 * M_PI;
        for (int it = 0; it < 100 && !equator; ++it) {
            double sh = std::sin(0.5 * th);
            double y = 2.0 * sh * sh;
            double P, D;
            legendre_y(n, y, &P, &D);
            // d/dtheta P_n(cos theta) = n (D_n - y P_n) / sin(theta)
            double step = P * std::sin(th) / (n * (D - y * P));
            th -= step;
            if (std::fabs(step) <= 1e-16 * th) break;
        }
        double sh = std::sin(0.5 * th);
        double y = 2.0 * sh * sh;
        double P, D;
        legendre_y(n, y, &P, &D);
        double st = std::sin(th);
        double den = n * (D - y * P);
        theta[i] = th;
        x[i] = equator ? 0.0 : std::cos(th);
        s[i] = st;
        w[i] = 2.0 * st * st / (den * den);
        // mirror node in the southern hemisphere
        int j = n - 1 - i;
        if (j != i) {
            theta[j] = M_PI - th;
            x[j] = -x[i];
            s[j] = st;
            w[j] = w[i];
        }
    }
}

void legendre_column(int Kmax, int m, int np, const double* x, const double* s, double* out) {
    const double two200 = std::ldexp(1.0, 200), inv200 = std::ldexp(1.0, -200);
    std::vector<double> epsK(Kmax + 2, 0.0);
    for (int K = m + 1; K <= Kmax + 1; ++K)
        epsK[K] = std::sqrt((double(K) * K - double(m) * m) / (4.0 * K * K - 1.0));
    for (int p = 0; p < np; ++p) {
        // diagonal Pt_m^m = (-1)^m sqrt((2m+1)/(4 pi) prod (2k-1)/(2k)) sin^m
        double mant = 1.0 / std::sqrt(4.0 * M_PI);
        long e = 0;
        for (int k = 1; k <= m; ++k) {
            int e2;
            mant = -std::sqrt((2.0 * k + 1.0) / (2.0 * k)) * s[p] * mant;
            mant = std::frexp(mant, &e2);
            e += e2;
        }
        double p2 = 0.0, p1 = mant;
        auto emit = [&](int K, double v, long ex) {
            double r = ex < -2000 ? 0.0 : std::ldexp(v, int(ex));
            out[size_t(K - m) * np + p] = r;
        };
        emit(m, p1, e);
        for (int K = m + 1; K <= Kmax; ++K) {
            double p0 = (K == m + 1) ? std::sqrt(2.0 * m + 3.0) * x[p] * p1
                                     : (x[p] * p1 - epsK[K - 1] * p2) / epsK[K];
            p2 = p1;
            p1 = p0;
            if (std::fabs(p1) > two200) {
                p1 *= inv200;
                p2 *= inv200;
                e += 200;
            }
            emit(K, p1, e);
        }
    }
}

void legendre_table_syn(int N, int nh, const double* x, const double* s, double* out) {
    unsigned nt = std::thread::hardware_concurrency();
    if (nt == 0) nt = 4;
    if (nt > 64) nt = 64;
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nt; ++t) {
        pool.emplace_back([=]() {
            std::vector<double> col;
            // interleave orders so that every thread gets light and heavy columns
            for (int m = int(t); m <= N; m += int(nt)) {
                int cnt = ext_count(N, m);
                col.resize(size_t(cnt) * nh);
                legendre_column(N + 1, m, nh, x, s, col.data());
                for (int K = m; K <= N + 1; ++K) {
                    double* dst = out + size_t(ext_row(N, m, K)) * nh;
                    const double* src = col.data() + size_t(K - m) * nh;
                    for (int p = 0; p < nh; ++p) dst[p] = src[p];
                }
            }
        });
    }
    for (auto& th : pool) th.join();
}

bool make_fft_plan(int n, FFTPlan* p) {
    p->n = n;
    p->nstages = 0;
    int r = n;
    while (r % 8 == 0) { p->radix[p->nstages++] = 8; r /= 8; }
    while (r % 4 == 0) { p->radix[p->nstages++] = 4; r /= 4; }
    while (r % 2 == 0) { p->radix[p->nstages++] = 2; r /= 2; }
    while (r % 3 == 0) { p->radix[p->nstages++] = 3; r /= 3; }
    return r == 1 && p->nstages <= 24;
}

}  // namespace sph
