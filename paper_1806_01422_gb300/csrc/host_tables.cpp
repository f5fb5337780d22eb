// Host-side tables of the spectral-element operators (arXiv:1806.01422, Sec. 3.2):
// Gauss-Lobatto-Legendre nodes and weights, the collocation derivative matrix,
// and the four 1D matrices the element kernels contract with.
#include "host_tables.h"

#include <cmath>

namespace semh {

// P_N and P_N' at x by the Legendre recurrence.
static void legendre_and_derivative(int N, double x, double& p, double& dp) {
    double p0 = 1.0, p1 = x;
    if (N == 0) { p = 1.0; dp = 0.0; return; }
    for (int k = 1; k < N; ++k) {
        const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    p = p1;
    // (1 - x^2) P_N' = N (P_{N-1} - x P_N); at x = +-1 use P_N'(+-1) = (+-1)^{N+1} N(N+1)/2
    if (std::fabs(1.0 - x * x) < 1e-300) dp = (x > 0 ? 1.0 : (N % 2 ? 1.0 : -1.0)) * 0.5 * N * (N + 1);
    else dp = N * (p0 - x * p1) / (1.0 - x * x);
}

// GLL nodes (ascending) and weights: endpoints plus the roots of P_N', the
// latter by Newton's method on P_N' using P_N'' from Legendre's equation
// (1 - x^2) P'' = 2x P' - N(N+1) P, started from Chebyshev-Lobatto points.
// The node set is symmetrised so that x[n-1-i] = -x[i] exactly.
void gll(int N, std::vector<double>& x, std::vector<double>& w) {
    const int n = N + 1;
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    x[0] = -1.0;
    x[N] = 1.0;
    for (int i = 1; i < N; ++i) {
        double r = -std::cos(M_PI * i / N);
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre_and_derivative(N, r, p, dp);
            const double d2p = (2.0 * r * dp - N * (N + 1.0) * p) / (1.0 - r * r);
            const double step = dp / d2p;
            r -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        x[i] = r;
    }
    for (int i = 0; i < n / 2; ++i) {
        const double s = 0.5 * (x[n - 1 - i] - x[i]);
        x[i] = -s;
        x[n - 1 - i] = s;
    }
    if (n % 2) x[n / 2] = 0.0;
    for (int i = 0; i < n; ++i) {
        double p, dp;
        legendre_and_derivative(N, x[i], p, dp);
        w[i] = 2.0 / (N * (N + 1.0) * p * p);
    }
    for (int i = 0; i < n / 2; ++i) {
        const double s = 0.5 * (w[i] + w[n - 1 - i]);
        w[i] = w[n - 1 - i] = s;
    }
}

// Collocation derivative D[i][j] = l_j'(x_i) by barycentric interpolation:
// lambda_j = 1 / prod_{k != j} (x_j - x_k), D_ij = (lambda_j / lambda_i) / (x_i - x_j),
// D_ii = -sum_{j != i} D_ij (rows annihilate constants).  Centro-antisymmetry
// D[n-1-i][n-1-j] = -D[i][j] holds exactly for symmetric nodes and is imposed.
void derivative(const std::vector<double>& x, std::vector<double>& D) {
    const int n = (int)x.size();
    std::vector<double> lam(n, 1.0);
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k)
            if (k != j) lam[j] *= (x[j] - x[k]);
    for (int j = 0; j < n; ++j) lam[j] = 1.0 / lam[j];
    D.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        double diag = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const double v = (lam[j] / lam[i]) / (x[i] - x[j]);
            D[(size_t)i * n + j] = v;
            diag -= v;
        }
        D[(size_t)i * n + i] = diag;
    }
    std::vector<double> S(D);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            S[(size_t)i * n + j] = 0.5 * (D[(size_t)i * n + j] - D[(size_t)(n - 1 - i) * n + (n - 1 - j)]);
    D.swap(S);
}

// Element-kernel matrices (row-major n x n, in this order):
//   Dg  = (2/h) Dhat                                  (centro-antisymmetric)
//   Sv  = -nu (2/h)^2 W^-1 Dhat^T W Dhat              (centro-symmetric)
//   Gv  = nu (2/h) W Dhat W^-1                        (centro-antisymmetric)
//         so that Dd Gv = -nu (2/h)^2 Dhat^T W Dhat W^-1 = Sv^T: the viscous term of
//         J^T and its advective flux share one divergence, Dd (Gv z + u o z)
//   Dd  = -(2/h) Dhat^T                               (centro-antisymmetric)
// Sv is symmetrised exactly, A[i][j] = A[n-1-i][n-1-j], and Gv antisymmetrised,
// A[i][j] = -A[n-1-i][n-1-j].
void kernel_matrices(const std::vector<double>& w, const std::vector<double>& Dh, double h, double nu,
                     std::vector<double>& mats) {
    const int n = (int)w.size();
    const double s = 2.0 / h;
    mats.assign((size_t)4 * n * n, 0.0);
    double* Dg = mats.data();
    double* Sv = Dg + n * n;
    double* Gv = Sv + n * n;
    double* Dd = Gv + n * n;
    std::vector<double> K((size_t)n * n, 0.0);  // Dhat^T W Dhat
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += Dh[(size_t)k * n + i] * w[k] * Dh[(size_t)k * n + j];
            K[(size_t)i * n + j] = acc;
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            Dg[i * n + j] = s * Dh[(size_t)i * n + j];
            Sv[i * n + j] = -nu * s * s * K[(size_t)i * n + j] / w[i];
            Gv[i * n + j] = nu * s * w[i] * Dh[(size_t)i * n + j] / w[j];
            Dd[i * n + j] = -s * Dh[(size_t)j * n + i];
        }
    for (double* A : {Sv, Gv}) {
        const double sign = A == Sv ? 1.0 : -1.0;
        std::vector<double> S(A, A + n * n);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                A[i * n + j] = 0.5 * (S[(size_t)i * n + j] + sign * S[(size_t)(n - 1 - i) * n + (n - 1 - j)]);
    }
}

}  // namespace semh

// ------------------------------------------------------------ binomial schedule
// P(1, s) = 0, P(l, 0) = l(l-1)/2 (restart from the stored state for every step),
// P(l, s) = min over the first split m of  m + P(l-m, s-1) + P(m, s):
// advance m steps, store that state, reverse the tail with one slot fewer, then
// reverse the head with the slot freed again.  Ties keep the largest m, which
// advances furthest while the forward sweep is storing (fewer later restarts).
namespace semh {

CkptPlanner::CkptPlanner(int L, int S) : L_(L < 1 ? 1 : L), S_(S < 0 ? 0 : S) {
    P_.assign((size_t)(L_ + 1) * (S_ + 1), 0);
    M_.assign((size_t)(L_ + 1) * (S_ + 1), 0);
    for (int l = 2; l <= L_; ++l) {
        P_[idx(l, 0)] = (long long)l * (l - 1) / 2;
        for (int s = 1; s <= S_; ++s) {
            long long best = -1;
            int bm = 1;
            for (int m = 1; m < l; ++m) {
                const long long c = m + P_[idx(l - m, s - 1)] + P_[idx(m, s)];
                if (best < 0 || c <= best) { best = c; bm = m; }
            }
            P_[idx(l, s)] = best;
            M_[idx(l, s)] = bm;
        }
    }
}

std::vector<int> CkptPlanner::forward_checkpoints(int nsteps, int slots) const {
    std::vector<int> pos{0};
    int a = 0, l = nsteps, free = slots - 1;
    while (l > 1 && free > 0) {
        const int m = split(l, free);
        a += m;
        l -= m;
        free -= 1;
        pos.push_back(a);
    }
    return pos;
}

static void rev(const CkptPlanner& P, int a, int l, int free, int slot, bool fresh,
                std::vector<CkptAction>& out) {
    if (l == 1) {
        out.push_back({CkptAction::RESTORE, slot, a});
        out.push_back({CkptAction::REVERSE, a, a});
        return;
    }
    if (free == 0) {
        for (int k = l - 1; k >= 0; --k) {
            out.push_back({CkptAction::RESTORE, slot, a});
            if (k > 0) out.push_back({CkptAction::ADVANCE, k, a + k});
            out.push_back({CkptAction::REVERSE, a + k, a + k});
        }
        return;
    }
    const int m = P.split(l, free);
    if (!fresh) {
        out.push_back({CkptAction::RESTORE, slot, a});
        out.push_back({CkptAction::ADVANCE, m, a + m});
        out.push_back({CkptAction::STORE, slot + 1, a + m});
    }
    rev(P, a + m, l - m, free - 1, slot + 1, fresh, out);
    rev(P, a, m, free, slot, false, out);
}

std::vector<CkptAction> CkptPlanner::backward_actions(int nsteps, int slots) const {
    std::vector<CkptAction> out;
    rev(*this, 0, nsteps, slots - 1, 0, true, out);
    return out;
}

}  // namespace semh
