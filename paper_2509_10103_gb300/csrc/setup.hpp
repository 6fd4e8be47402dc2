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

// Banded LU factor tables are tiled for the device solver: k is grouped in
// tiles of kTileK consecutive values (one tile = the systems of one solver
// block), and within a (matrix, tile) the forward-sweep columns [0, nc1) of
// every row come first, then the backward-sweep columns [nc1, kBand):
//   table[mat][tile][part 0: j][e < nc1][kk] , [part 1: j][e - nc1][kk]
// so a run of consecutive rows of one sweep is one contiguous piece.
constexpr int kTileK = 32;
inline size_t fac_index(int mat, int k, int j, int e, int nr, int ntile, int nc1) {
    const size_t tile = ((size_t)mat * ntile + k / kTileK) * (size_t)nr * kBand * kTileK;
    const size_t in = e < nc1 ? ((size_t)j * nc1 + e) * kTileK
                              : (size_t)nr * nc1 * kTileK + ((size_t)j * (kBand - nc1) + (e - nc1)) * kTileK;
    return tile + in + k % kTileK;
}
constexpr int kNc1Direct = kLo;          // A x = b rows: l (4) | 1/diag, U (9)
constexpr int kNc1Transposed = kUp + 1;  // A^T x = b rows: U^T (8), 1/diag | L^T (4)

// Everything the device needs, laid out for coalesced access across k.
struct HostOps {
    Dims d;
    Physics ph;
    std::vector<double> r, invr, W;            // [nr]
    std::vector<double> D1, D2;                 // [2 parity][nr][kBand], parity 0 even, 1 odd
    std::vector<double> Lb;                     // [M+2][nr][kBand]  D2 + D1/r - m^2/r^2 (no kz^2)
    // Banded LU factors in the tiled layout of fac_index (ntile tiles of k,
    // zeros beyond nk).  Row layout "lower | 1/diag | upper" for a two-sweep solve:
    //   facH/facP  (A x = b):   l_{j,j-4..j-1}, 1/U_jj, U_{j,j+1..j+8}    (nc1 = kNc1Direct)
    //   facHT/facPT (A^T x = b): U_{j-8..j-1,j}, 1/U_jj, L_{j+1..j+4,j}  (nc1 = kNc1Transposed)
    int ntile = 0;
    std::vector<double> facH, facHT;            // M+2 matrices (per |m'|, k)  Helmholtz
    std::vector<double> facP, facPT;            // M+1 matrices (per |m|, k)   pressure
    std::vector<double> infl;                   // [nm][3][nr][nk] influence response, pre-scaled by -1/delta
    std::vector<double> fluxg;                  // [nr] flux response of mode (0,0)
    double flux_inv = 0;                        // 1 / sum_j W_j g_j
    std::vector<std::complex<double>> Uh, dUh;  // [nr] oscillatory base-flow profiles
    double omega = 0;                           // pulsation angular frequency Wo^2/Re
};

int parity_index(int m);  // 0 when m is even, 1 when odd

// Builds grid, weights and finite differences (Re-independent part).
bool build_grid(HostOps& h, std::string& err);
// Builds base flow, banded LU factors, influence and flux vectors.
// reuse_pressure: keep h.facP / h.facPT when they already have this grid's
// size (they depend on the grid only, not on Re or dt).
bool build_operators(HostOps& h, std::string& err, bool reuse_pressure = false);

// Bessel J_nu of complex argument by its power series.
std::complex<double> bessel_j(int nu, std::complex<double> z);

// Factors for the orthogonal projection onto admissible fields (no slip,
// discretely solenoidal; Section 2.2 constraints) in the energy inner product.
// For mode (m, k) != (0, 0), with the wall values removed, the constraint
// C x = D_r x_r + (i m / r) x_theta + i k_z x_z = 0 at every r_j gives the
// real symmetric positive definite system
//   S = D_r W^-1 D_r^T + diag((m^2 / r^2 + k_z^2) / W)  (rows j >= 1 for the diagonal),
// D_r = D1 (parity of m + 1) + 1/r over the columns j >= 1, banded with
// half-bandwidth kProjBand.  L holds its banded Cholesky factor per (|m|, k):
// [|m| = 0..M][k][j][e], e = i - j + kProjBand for i = j - kProjBand .. j - 1,
// and e = kProjBand holding 1 / L_jj.
constexpr int kProjBand = 12;
bool build_projection(const HostOps& h, std::vector<double>& L, std::string& err);

// Binomial checkpointing (Section 2.5).
long long binom_beta(int s, long long t);
int revolve_repetitions(long long nsteps, int snaps);
long long revolve_advances(long long nsteps, int snaps);

}  // namespace pnop
