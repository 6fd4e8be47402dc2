// Host construction of grid, quadrature, finite differences, banded LU
// factors, influence/flux responses and base-flow profiles (FP64).
//
// Section 2.4 (Keuchel & Avila): N_r Chebyshev points with optional
// relaxation, high-order radial finite differences, Fourier modes in theta
// and z, influence-matrix wall conditions, flux forcing f_z (Eq. 2.7).
// Eq. 2.3-2.4: steady profile plus the Sexl-Womersley oscillation.
#include "setup.hpp"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <random>
#include <thread>
#include <vector>

namespace pnop {

using cd = std::complex<double>;

int parity_index(int m) { return (m % 2 == 0) ? 0 : 1; }

// ---------------------------------------------------------------- grid
static void radial_points(int nr, double stretch, std::vector<double>& r) {
    r.resize(nr);
    const double last = std::cos(M_PI * (nr - 1) / (2.0 * nr - 1.0));
    for (int j = 0; j < nr; ++j) {
        double x = std::cos(M_PI * j / (2.0 * nr - 1.0));
        double rho = 1.0 - j * (1.0 - last) / (nr - 1.0);
        r[j] = (1.0 - stretch) * x + stretch * rho;
    }
    r[0] = 1.0;
}

// Dense LU with partial pivoting (long double), solves A x = b in place.
static bool dense_solve(int n, std::vector<long double>& A, std::vector<long double>& b) {
    std::vector<int> piv(n);
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int i = c + 1; i < n; ++i)
            if (std::fabs(A[i * n + c]) > std::fabs(A[p * n + c])) p = i;
        if (A[p * n + c] == 0) return false;
        if (p != c) {
            for (int k = 0; k < n; ++k) std::swap(A[p * n + k], A[c * n + k]);
            std::swap(b[p], b[c]);
        }
        for (int i = c + 1; i < n; ++i) {
            long double f = A[i * n + c] / A[c * n + c];
            if (f == 0) continue;
            for (int k = c; k < n; ++k) A[i * n + k] -= f * A[c * n + k];
            b[i] -= f * b[c];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        long double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= A[i * n + k] * b[k];
        b[i] = s / A[i * n + i];
    }
    return true;
}

// Quadrature for int_0^1 f r dr exact when f is a polynomial of degree < nr
// in s = r^2: half the interpolatory weights of int_0^1 ds on s_j = r_j^2,
// from the Chebyshev moment equations sum_j T_n(2 s_j - 1) w_j = mu_n.
static bool radial_quadrature(const std::vector<double>& r, std::vector<double>& W) {
    const int n = (int)r.size();
    std::vector<long double> A((size_t)n * n), b(n);
    for (int j = 0; j < n; ++j) {
        long double x = 2.0L * (long double)r[j] * (long double)r[j] - 1.0L;
        long double t0 = 1.0L, t1 = x;
        for (int k = 0; k < n; ++k) {
            long double tk = (k == 0) ? t0 : (k == 1 ? t1 : 0.0L);
            if (k >= 2) {
                tk = 2.0L * x * t1 - t0;
                t0 = t1;
                t1 = tk;
            }
            A[(size_t)k * n + j] = tk;
        }
    }
    for (int k = 0; k < n; ++k) b[k] = (k % 2 == 0) ? 1.0L / (1.0L - (long double)k * k) : 0.0L;
    if (!dense_solve(n, A, b)) return false;
    W.resize(n);
    for (int j = 0; j < n; ++j) W[j] = (double)(0.5L * b[j]);
    return true;
}

// Weights of the d-th derivative at x0 from 9 nodes: exactness on (x-x0)^p,
// p = 0..8, solved as a Vandermonde system in the scaled offsets.
static bool fd_weights(double x0, const double* x, int d, double* w) {
    const int n = kStencil;
    long double h = 0;
    for (int i = 0; i < n; ++i) h = std::max(h, std::fabs((long double)x[i] - x0));
    std::vector<long double> A((size_t)n * n), b(n, 0.0L);
    for (int p = 0; p < n; ++p)
        for (int i = 0; i < n; ++i) A[(size_t)p * n + i] = std::pow(((long double)x[i] - x0) / h, p);
    long double fact = 1;
    for (int q = 2; q <= d; ++q) fact *= q;
    b[d] = fact;
    if (!dense_solve(n, A, b)) return false;
    for (int i = 0; i < n; ++i) w[i] = (double)(b[i] / std::pow(h, d));
    return true;
}

bool build_grid(HostOps& h, std::string& err) {
    const Dims& d = h.d;
    const int nr = d.nr;
    radial_points(nr, d.stretch, h.r);
    h.invr.resize(nr);
    for (int j = 0; j < nr; ++j) h.invr[j] = 1.0 / h.r[j];
    if (!radial_quadrature(h.r, h.W)) {
        err = "radial quadrature system is singular";
        return false;
    }
    for (int j = 0; j < nr; ++j)
        if (!(h.W[j] > 0)) {
            err = "radial quadrature weight is not positive (stretch too large?)";
            return false;
        }
    // finite differences on the mirrored grid {r} U {-r}; a mirrored node
    // carries parity * f(r_i).  Rows near the wall are one-sided.
    std::vector<double> ext(2 * nr);
    for (int e = 0; e < nr; ++e) ext[e] = h.r[e];
    for (int e = nr; e < 2 * nr; ++e) ext[e] = -h.r[2 * nr - 1 - e];
    h.D1.assign((size_t)2 * nr * kBand, 0.0);
    h.D2.assign((size_t)2 * nr * kBand, 0.0);
    for (int j = 0; j < nr; ++j) {
        int lo = std::min(std::max(j - kStencil / 2, 0), 2 * nr - kStencil);
        double w1[kStencil], w2[kStencil];
        if (!fd_weights(h.r[j], &ext[lo], 1, w1) || !fd_weights(h.r[j], &ext[lo], 2, w2)) {
            err = "finite-difference system is singular";
            return false;
        }
        for (int pi = 0; pi < 2; ++pi) {
            const double par = pi == 0 ? 1.0 : -1.0;
            for (int t = 0; t < kStencil; ++t) {
                int e = lo + t;
                int col = e < nr ? e : 2 * nr - 1 - e;
                double sg = e < nr ? 1.0 : par;
                int s = col - j + kLo;
                if (s < 0 || s >= kBand) {
                    err = "stencil outside the stored band";
                    return false;
                }
                h.D1[((size_t)pi * nr + j) * kBand + s] += sg * w1[t];
                h.D2[((size_t)pi * nr + j) * kBand + s] += sg * w2[t];
            }
        }
    }
    return true;
}

// ---------------------------------------------------------------- Bessel / base flow
cd bessel_j(int nu, cd z) {
    cd half = 0.5 * z;
    cd term = 1.0;
    for (int i = 0; i < nu; ++i) term *= half / double(i + 1);
    cd sum = term;
    cd q = -half * half;
    for (int k = 1; k < 400; ++k) {
        term *= q / double(k * (k + nu));
        sum += term;
        if (std::abs(term) <= 1e-18 * std::max(std::abs(sum), 1e-300)) break;
    }
    return sum;
}

static void base_profiles(HostOps& h) {
    const int nr = h.d.nr;
    h.Uh.assign(nr, cd(0, 0));
    h.dUh.assign(nr, cd(0, 0));
    h.omega = h.ph.Wo * h.ph.Wo / h.ph.Re;
    if (h.ph.A == 0.0) return;
    const cd kappa = std::polar(h.ph.Wo, 0.75 * M_PI);
    const cd j0k = bessel_j(0, kappa), j1k = bessel_j(1, kappa);
    // bulk of the oscillation = (A/2) sin(omega t): B (1 - 2 J1/(kappa J0)) = -i A / 2
    const cd B = cd(0.0, -0.5 * h.ph.A) / (1.0 - 2.0 * j1k / (kappa * j0k));
    for (int j = 0; j < nr; ++j) {
        cd kr = kappa * h.r[j];
        h.Uh[j] = B * (1.0 - bessel_j(0, kr) / j0k);
        h.dUh[j] = B * kappa * bessel_j(1, kr) / j0k;
    }
}

// ---------------------------------------------------------------- banded LU
// Band row j holds columns j-4 .. j+8 at offsets 0..12.
struct Band {
    int n;
    std::vector<double> a;  // [n][kBand]
    double& at(int j, int col) { return a[(size_t)j * kBand + (col - j + kLo)]; }
    double get(int j, int col) const {
        int s = col - j + kLo;
        if (s < 0 || s >= kBand || col < 0 || col >= n) return 0.0;
        return a[(size_t)j * kBand + s];
    }
};

// Doolittle LU without pivoting.  Output per row: l[0..3] (columns j-4..j-1),
// 1/U_jj, U_{j,j+1..j+8}.
static bool band_lu(const Band& A, std::vector<double>& f, double& growth) {
    const int n = A.n;
    std::vector<double> U((size_t)n * (kUp + 1), 0.0);  // U[j][0..8] = U_{j,j..j+8}
    f.assign((size_t)n * kBand, 0.0);
    double amax = 0, umax = 0;
    for (double v : A.a) amax = std::max(amax, std::fabs(v));
    for (int j = 0; j < n; ++j) {
        double row[kLo + kUp + 1];  // columns j-4 .. j+8
        for (int s = 0; s < kBand; ++s) row[s] = A.get(j, j - kLo + s);
        for (int i = std::max(0, j - kLo); i < j; ++i) {
            double piv = U[(size_t)i * (kUp + 1)];
            double l = row[i - j + kLo] / piv;
            row[i - j + kLo] = 0.0;
            for (int c = i + 1; c <= std::min(n - 1, i + kUp); ++c) {
                int s = c - j + kLo;
                if (s >= kBand) {
                    if (U[(size_t)i * (kUp + 1) + (c - i)] != 0.0 && l != 0.0) return false;  // fill beyond band
                    continue;
                }
                row[s] -= l * U[(size_t)i * (kUp + 1) + (c - i)];
            }
            f[(size_t)j * kBand + (i - (j - kLo))] = l;
        }
        if (row[kLo] == 0.0) return false;
        for (int c = 0; c <= kUp; ++c) {
            double v = (j + c < n) ? row[kLo + c] : 0.0;
            U[(size_t)j * (kUp + 1) + c] = v;
            umax = std::max(umax, std::fabs(v));
        }
        f[(size_t)j * kBand + kLo] = 1.0 / row[kLo];
        for (int c = 1; c <= kUp; ++c) f[(size_t)j * kBand + kLo + c] = U[(size_t)j * (kUp + 1) + c];
    }
    growth = umax / std::max(amax, 1e-300);
    return true;
}

// Solve with factors f (real RHS, in place).
static void band_solve(int n, const std::vector<double>& f, std::vector<double>& x) {
    for (int j = 0; j < n; ++j) {
        double s = x[j];
        for (int e = 0; e < kLo; ++e) {
            int c = j - kLo + e;
            if (c >= 0) s -= f[(size_t)j * kBand + e] * x[c];
        }
        x[j] = s;
    }
    for (int j = n - 1; j >= 0; --j) {
        double s = x[j];
        for (int e = 1; e <= kUp; ++e) {
            int c = j + e;
            if (c < n) s -= f[(size_t)j * kBand + kLo + e] * x[c];
        }
        x[j] = s * f[(size_t)j * kBand + kLo];
    }
}

static double band_backward_error(const Band& A, const std::vector<double>& f, unsigned seed) {
    const int n = A.n;
    std::mt19937_64 g(seed);
    std::uniform_real_distribution<double> U(-1, 1);
    std::vector<double> b(n), x;
    for (int j = 0; j < n; ++j) b[j] = U(g);
    x = b;
    band_solve(n, f, x);
    double rmax = 0, amax = 0, xmax = 0;
    for (int j = 0; j < n; ++j) {
        double s = -b[j], arow = 0;
        for (int c = std::max(0, j - kLo); c <= std::min(n - 1, j + kUp); ++c) {
            s += A.get(j, c) * x[c];
            arow += std::fabs(A.get(j, c));
        }
        rmax = std::max(rmax, std::fabs(s));
        amax = std::max(amax, arow);
        xmax = std::max(xmax, std::fabs(x[j]));
    }
    return rmax / (amax * xmax + 1e-300);
}

static void scatter_factors(std::vector<double>& dst, int mat, int k, int nr, int ntile, int nc1,
                            const std::vector<double>& f) {
    for (int j = 0; j < nr; ++j)
        for (int e = 0; e < kBand; ++e) dst[fac_index(mat, k, j, e, nr, ntile, nc1)] = f[(size_t)j * kBand + e];
}

static void gather_factors(const std::vector<double>& src, int mat, int k, int nr, int ntile, int nc1,
                           std::vector<double>& f) {
    f.resize((size_t)nr * kBand);
    for (int j = 0; j < nr; ++j)
        for (int e = 0; e < kBand; ++e) f[(size_t)j * kBand + e] = src[fac_index(mat, k, j, e, nr, ntile, nc1)];
}

// Row-local coefficients of A^T = U^T L^T from the factors of A: row j holds
// U_{j-8+e, j} (e = 0..7, oldest first), 1/U_jj, L_{j+1+e, j} (e = 0..3).
static std::vector<double> transpose_factors(int nr, const std::vector<double>& f) {
    std::vector<double> t((size_t)nr * kBand, 0.0);
    for (int j = 0; j < nr; ++j) {
        for (int e = 0; e < 8; ++e) {
            const int i = j - 8 + e;  // U_{i, j} = f[i][4 + (j - i)]
            if (i >= 0) t[(size_t)j * kBand + e] = f[(size_t)i * kBand + kLo + (j - i)];
        }
        t[(size_t)j * kBand + 8] = f[(size_t)j * kBand + kLo];
        for (int e = 0; e < 4; ++e) {
            const int i = j + 1 + e;  // L_{i, j} = f[i][j - i + 4]
            if (i < nr) t[(size_t)j * kBand + 9 + e] = f[(size_t)i * kBand + (j - i + kLo)];
        }
    }
    return t;
}

static Band laplacian_band(const HostOps& h, int mabs, double kz) {
    const int nr = h.d.nr;
    Band L{nr, std::vector<double>((size_t)nr * kBand, 0.0)};
    for (int j = 0; j < nr; ++j)
        for (int s = 0; s < kBand; ++s) L.a[(size_t)j * kBand + s] = h.Lb[((size_t)mabs * nr + j) * kBand + s];
    for (int j = 0; j < nr; ++j) L.at(j, j) -= kz * kz;
    return L;
}

static Band helmholtz_band(const HostOps& h, int mabs, double kz) {
    const int nr = h.d.nr;
    Band A = laplacian_band(h, mabs, kz);
    const double c = -1.0 / (2.0 * h.ph.Re);
    for (double& v : A.a) v *= c;
    for (int j = 0; j < nr; ++j) A.at(j, j) += 1.0 / h.ph.dt;
    for (int s = 0; s < kBand; ++s) A.a[s] = 0.0;
    A.at(0, 0) = 1.0;  // Dirichlet row
    return A;
}

static Band pressure_band(const HostOps& h, int mabs, double kz) {
    const int nr = h.d.nr;
    Band A = laplacian_band(h, mabs, kz);
    const int pi = parity_index(mabs);
    for (int s = 0; s < kBand; ++s) A.a[s] = h.D1[((size_t)pi * nr + 0) * kBand + s];  // Neumann row
    return A;
}

// fn(k) for k = 0..n-1 on up to 16 host threads; fn touches only data of its own k.
template <class F> static void parallel_k(int n, F&& fn) {
    const int T = std::max(1, std::min<int>({n, 16, (int)std::max(1u, std::thread::hardware_concurrency())}));
    if (T == 1) {
        for (int k = 0; k < n; ++k) fn(k, 0);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t)
        th.emplace_back([&, t] {
            for (int k = t; k < n; k += T) fn(k, t);
        });
    for (auto& x : th) x.join();
}

bool build_operators(HostOps& h, std::string& err, bool reuse_pressure) {
    const Dims& d = h.d;
    const int nr = d.nr, nk = d.nk, M = d.M;
    if (!(h.ph.Re > 0) || !(h.ph.dt > 0)) {
        err = "Re and dt must be positive";
        return false;
    }
    base_profiles(h);
    // L band for |m'| = 0..M+1: D2 + D1/r - m'^2/r^2, parity of m'
    h.Lb.assign((size_t)(M + 2) * nr * kBand, 0.0);
    for (int ma = 0; ma <= M + 1; ++ma) {
        const int pi = parity_index(ma);
        for (int j = 0; j < nr; ++j) {
            for (int s = 0; s < kBand; ++s) {
                size_t src = ((size_t)pi * nr + j) * kBand + s;
                h.Lb[((size_t)ma * nr + j) * kBand + s] = h.D2[src] + h.invr[j] * h.D1[src];
            }
            h.Lb[((size_t)ma * nr + j) * kBand + kLo] -= (double)ma * ma * h.invr[j] * h.invr[j];
        }
    }
    const int nt = h.ntile = (nk + kTileK - 1) / kTileK;
    const int D = kNc1Direct, T = kNc1Transposed;
    const size_t pressure_size = (size_t)(M + 1) * nt * nr * kBand * kTileK;
    // the pressure factors depend on the grid only: a caller that built them
    // for this grid before may keep them
    const bool pressure = !(reuse_pressure && h.facP.size() == pressure_size && h.facPT.size() == pressure_size);
    h.facH.assign((size_t)(M + 2) * nt * nr * kBand * kTileK, 0.0);
    h.facHT.assign(h.facH.size(), 0.0);
    if (pressure) {
        h.facP.assign(pressure_size, 0.0);
        h.facPT.assign(pressure_size, 0.0);
    }
    // every k owns its own factor entries, so the k loop runs on host threads
    std::vector<double> worst_t(16, 0.0);
    std::vector<int> fail_t(16, 0);
    parallel_k(nk, [&](int k, int t) {
        std::vector<double> f;
        double growth = 0;
        const double kz = 2.0 * M_PI * k / d.Lz;
        for (int ma = 0; ma <= M + 1; ++ma) {
            Band A = helmholtz_band(h, ma, kz);
            if (!band_lu(A, f, growth)) {
                fail_t[t] = 1;
                return;
            }
            worst_t[t] = std::max(worst_t[t], band_backward_error(A, f, 1234u + ma * 977u + k));
            scatter_factors(h.facH, ma, k, nr, nt, D, f);
            scatter_factors(h.facHT, ma, k, nr, nt, T, transpose_factors(nr, f));
        }
        if (!pressure) return;
        for (int ma = 0; ma <= M; ++ma) {
            if (ma == 0 && k == 0) {
                // singular Neumann problem of the mean mode: never used (p = 0)
                std::vector<double> id((size_t)nr * kBand, 0.0);
                for (int j = 0; j < nr; ++j) id[(size_t)j * kBand + kLo] = 1.0;
                scatter_factors(h.facP, ma, k, nr, nt, D, id);
                scatter_factors(h.facPT, ma, k, nr, nt, T, transpose_factors(nr, id));
                continue;
            }
            Band A = pressure_band(h, ma, kz);
            if (!band_lu(A, f, growth)) {
                fail_t[t] = 2;
                return;
            }
            worst_t[t] = std::max(worst_t[t], band_backward_error(A, f, 4321u + ma * 131u + k));
            scatter_factors(h.facP, ma, k, nr, nt, D, f);
            scatter_factors(h.facPT, ma, k, nr, nt, T, transpose_factors(nr, f));
        }
    });
    double worst = 0;
    for (int t = 0; t < 16; ++t) {
        if (fail_t[t]) {
            err = fail_t[t] == 1 ? "Helmholtz band LU failed" : "pressure band LU failed";
            return false;
        }
        worst = std::max(worst, worst_t[t]);
    }
    std::vector<double> f, fac_tmp;
    double growth = 0;
    if (!(worst < 1e-12)) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "banded LU without pivoting is unstable here (backward error %.3g)", worst);
        err = buf;
        return false;
    }
    // influence responses: phi solves the pressure problem with a unit wall
    // datum, h the Helmholtz response to -grad(phi) with u = 0 at the wall;
    // stored scaled by -1/delta, delta = d/dr(h_r) at the wall.
    h.infl.assign((size_t)d.nm * nk * 3 * nr, 0.0);
    std::vector<int> zero_t(16, 0);
    parallel_k(nk, [&](int k, int t) {
        std::vector<double> f, fac_tmp;
        const double kz = 2.0 * M_PI * k / d.Lz;
        for (int im = 0; im < d.nm; ++im) {
            const int m = im - M;
            if (m == 0 && k == 0) continue;
            const int ma = std::abs(m);
            gather_factors(h.facP, ma, k, nr, nt, D, f);  // factors computed above
            std::vector<double> phi(nr, 0.0);
            phi[0] = 1.0;
            band_solve(nr, f, phi);
            const int pp = parity_index(m);
            std::vector<double> dphi(nr, 0.0);
            for (int j = 0; j < nr; ++j)
                for (int c = std::max(0, j - kLo); c <= std::min(nr - 1, j + kUp); ++c)
                    dphi[j] += h.D1[((size_t)pp * nr + j) * kBand + (c - j + kLo)] * phi[c];
            std::vector<double> fp(nr), fm(nr), fz(nr);
            for (int j = 0; j < nr; ++j) {
                fp[j] = -dphi[j] + m * h.invr[j] * phi[j];
                fm[j] = -dphi[j] - m * h.invr[j] * phi[j];
                fz[j] = -kz * phi[j];  // imaginary part of -i kz phi
            }
            fp[0] = fm[0] = fz[0] = 0.0;
            gather_factors(h.facH, std::abs(m + 1), k, nr, nt, D, fac_tmp);
            band_solve(nr, fac_tmp, fp);
            gather_factors(h.facH, std::abs(m - 1), k, nr, nt, D, fac_tmp);
            band_solve(nr, fac_tmp, fm);
            gather_factors(h.facH, ma, k, nr, nt, D, fac_tmp);
            band_solve(nr, fac_tmp, fz);
            std::vector<double> hr(nr), hti(nr);
            for (int j = 0; j < nr; ++j) {
                hr[j] = 0.5 * (fp[j] + fm[j]);
                hti[j] = -0.5 * (fp[j] - fm[j]);
            }
            const int pv = parity_index(m + 1);
            double delta = 0;
            for (int c = 0; c <= kUp && c < nr; ++c) delta += h.D1[((size_t)pv * nr + 0) * kBand + (c + kLo)] * hr[c];
            if (!(std::fabs(delta) > 1e-300) || !std::isfinite(delta)) {
                zero_t[t] = 1;
                return;
            }
            // k fastest: [im][component][j][k], so that the device reads it
            // coalesced across the k of a block
            double* out = &h.infl[(size_t)im * 3 * nr * nk + k];
            for (int j = 0; j < nr; ++j) {
                out[(size_t)j * nk] = -hr[j] / delta;
                out[((size_t)nr + j) * nk] = -hti[j] / delta;
                out[((size_t)2 * nr + j) * nk] = -fz[j] / delta;
            }
        }
    });
    for (int t = 0; t < 16; ++t)
        if (zero_t[t]) {
            err = "influence response has zero wall divergence";
            return false;
        }
    // flux response of mode (0,0): Helmholtz of u_z with unit forcing
    {
        Band Hz = helmholtz_band(h, 0, 0.0);
        band_lu(Hz, fac_tmp, growth);
        h.fluxg.assign(nr, 1.0);
        h.fluxg[0] = 0.0;
        band_solve(nr, fac_tmp, h.fluxg);
        double s = 0;
        for (int j = 0; j < nr; ++j) s += h.W[j] * h.fluxg[j];
        h.flux_inv = 1.0 / s;
    }
    return true;
}

// ---------------------------------------------------------------- checkpoint counts
long long binom_beta(int s, long long t) {
    if (t < 0) return 0;
    // C(s + t, s) = C(s + t, t) with saturation, over the shorter product
    const long long a = std::max<long long>(s, t), b = std::min<long long>(s, t);
    long double v = 1;
    for (long long i = 1; i <= b; ++i) {
        v = v * (long double)(a + i) / (long double)i;
        if (v > 4.0e18L) return (long long)4e18;
    }
    return (long long)(v + 0.5L);
}

bool build_projection(const HostOps& h, std::vector<double>& L, std::string& err) {
    const int nr = h.d.nr, M = h.d.M, nk = h.d.nk, B = kProjBand, W1 = B + 1;
    // A_par = D_r W^-1 D_r^T over the columns i >= 1, banded, for both parities
    std::vector<double> A[2];
    for (int par = 0; par < 2; ++par) {
        A[par].assign((size_t)nr * W1, 0.0);  // A[j][j' - j + B] for j' in [j - B, j]
        std::vector<std::vector<std::pair<int, double>>> col(nr);  // column i: (row j, D_r(j, i))
        for (int j = 0; j < nr; ++j)
            for (int e = 0; e < kBand; ++e) {
                const int i = j - kLo + e;
                if (i < 1 || i >= nr) continue;
                double v = h.D1[((size_t)par * nr + j) * kBand + e];
                if (i == j) v += h.invr[j];
                if (v != 0.0) col[i].push_back({j, v});
            }
        for (int i = 1; i < nr; ++i)
            for (auto& a : col[i])
                for (auto& b : col[i]) {
                    if (b.first > a.first) continue;
                    if (a.first - b.first > B) {
                        err = "admissible projection: divergence stencil wider than the factor band";
                        return false;
                    }
                    A[par][(size_t)a.first * W1 + (b.first - a.first + B)] += a.second * b.second / h.W[i];
                }
    }
    L.assign((size_t)(M + 1) * nk * nr * W1, 0.0);
    std::vector<double> S((size_t)nr * W1);
    for (int ma = 0; ma <= M; ++ma) {
        const int par = parity_index(ma + 1);
        for (int k = 0; k < nk; ++k) {
            if (ma == 0 && k == 0) continue;  // mean mode: diagonal constraints, no factor
            const double kz = 2.0 * M_PI * k / h.d.Lz;
            S = A[par];
            for (int j = 1; j < nr; ++j)
                S[(size_t)j * W1 + B] += ((double)ma * ma * h.invr[j] * h.invr[j] + kz * kz) / h.W[j];
            double* F = &L[(((size_t)ma * nk + k) * nr) * W1];
            for (int j = 0; j < nr; ++j) {
                for (int i = std::max(0, j - B); i <= j; ++i) {
                    double v = S[(size_t)j * W1 + (i - j + B)];
                    for (int q = std::max(0, j - B); q < i; ++q)
                        if (q >= i - B) v -= F[(size_t)j * W1 + (q - j + B)] * F[(size_t)i * W1 + (q - i + B)];
                    if (i < j) {
                        F[(size_t)j * W1 + (i - j + B)] = v * F[(size_t)i * W1 + B];
                    } else {
                        if (!(v > 0) || !std::isfinite(v)) {
                            err = "admissible projection: constraint system is not positive definite";
                            return false;
                        }
                        F[(size_t)j * W1 + B] = 1.0 / std::sqrt(v);
                    }
                }
            }
        }
    }
    return true;
}

int revolve_repetitions(long long nsteps, int snaps) {
    int r = 0;
    while (binom_beta(snaps, r) < nsteps) ++r;
    return r;
}

long long revolve_advances(long long nsteps, int snaps) {
    if (nsteps <= 1) return 0;
    int r = revolve_repetitions(nsteps, snaps);
    return (long long)r * nsteps - binom_beta(snaps + 1, r - 1);
}

}  // namespace pnop
