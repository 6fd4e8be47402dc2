// Host-side construction of the discrete operators (FP64, computed once per
// context).  Section 2.4 of Keuchel & Avila: Fourier-Galerkin in theta and z,
// high-order finite differences on Chebyshev radial points, influence-matrix
// wall conditions; Eq. 2.3-2.4 for the base flow.
#pragma once

#include <complex>
#include <string>
#include <vector>

namespace pnop {

constexpr int kBand = 13;   // stored band per row: columns j-4 .. j+8
constexpr int kLo = 4;      // lower bandwidth
constexpr int kUp = 8;      // upper bandwidth (one-sided wall stencils)
constexpr int kStencil = 9; // finite-difference points per row

struct Dims {
    int nr = 0, M = 0, K = 0;
    int nm = 0, nk = 0;       // 2M+1, K+1
    int nth = 0, nzp = 0;     // physical 3(M+1), 3(K+1)
    double Lz = 0, stretch = 0;
};

struct Physics {
    double Re = 0, Wo = 0, A = 0, dt = 0, tau0 = 0;
};

// Everything the device needs, laid out for coalesced access across k.
struct HostOps {
    Dims d;
    Physics ph;
    std::vector<double> r, invr, W;            // [nr]
    std::vector<double> D1, D2;                 // [2 parity][nr][kBand], parity 0 even, 1 odd
    std::vector<double> Lb;                     // [M+2][nr][kBand]  D2 + D1/r - m^2/r^2 (no kz^2)
    // Banded LU factors, k padded to nkp (a multiple of 32, zeros beyond nk).
    // Row layout "lower | 1/diag | upper" for a two-sweep solve:
    //   facH/facP  (A x = b):   l_{j,j-4..j-1}, 1/U_jj, U_{j,j+1..j+8}
    //   facHT/facPT (A^T x = b): U_{j-8..j-1,j}, 1/U_jj, L_{j+1..j+4,j}
    int nkp = 0;
    std::vector<double> facH, facHT;            // [M+2][nr][kBand][nkp]  Helmholtz (per |m'|, k)
    std::vector<double> facP, facPT;            // [M+1][nr][kBand][nkp]  pressure (per |m|, k)
    std::vector<double> infl;                   // [nm][nk][3][nr] influence response, pre-scaled by -1/delta
    std::vector<double> fluxg;                  // [nr] flux response of mode (0,0)
    double flux_inv = 0;                        // 1 / sum_j W_j g_j
    std::vector<std::complex<double>> Uh, dUh;  // [nr] oscillatory base-flow profiles
    double omega = 0;                           // pulsation angular frequency Wo^2/Re
};

int parity_index(int m);  // 0 when m is even, 1 when odd

// Builds grid, weights and finite differences (Re-independent part).
bool build_grid(HostOps& h, std::string& err);
// Builds base flow, banded LU factors, influence and flux vectors.
bool build_operators(HostOps& h, std::string& err);

// Bessel J_nu of complex argument by its power series.
std::complex<double> bessel_j(int nu, std::complex<double> z);

// Binomial checkpointing (Section 2.5).
long long binom_beta(int s, long long t);
int revolve_repetitions(long long nsteps, int snaps);
long long revolve_advances(long long nsteps, int snaps);

}  // namespace pnop
