// Host-side tables (GLL nodes, weights, derivative matrix, kernel matrices) and
// the binomial checkpoint planner.
#pragma once
#include <vector>

namespace semh {

void gll(int N, std::vector<double>& x, std::vector<double>& w);
void derivative(const std::vector<double>& x, std::vector<double>& D);
void kernel_matrices(const std::vector<double>& w, const std::vector<double>& Dh, double h, double nu,
                     std::vector<double>& mats);

// One primitive action of a checkpointed backward sweep.  `cur` is a working
// state buffer; slots hold stored states.
struct CkptAction {
    enum Kind { RESTORE = 0, ADVANCE = 1, STORE = 2, REVERSE = 3 } kind;
    int arg;    // RESTORE/STORE: slot; ADVANCE: number of steps; REVERSE: step index
    int step;   // step index of `cur` after the action (for checking)
};

// Optimal advance count P(l, s) for every l <= L, s <= S and the first split
// realising it (Sec. 5.3: revolve-optimal binomial checkpointing).
class CkptPlanner {
public:
    CkptPlanner(int L, int S);
    long long cost(int l, int s) const { return P_[idx(l, s)]; }
    int split(int l, int s) const { return M_[idx(l, s)]; }
    // Slot positions stored during the forward sweep (first descent of the
    // recursion from step 0 with `slots` slots, slot 0 = the initial state).
    std::vector<int> forward_checkpoints(int nsteps, int slots) const;
    // Actions of the backward sweep, given that forward_checkpoints() were stored.
    std::vector<CkptAction> backward_actions(int nsteps, int slots) const;

private:
    int L_, S_;
    std::vector<long long> P_;
    std::vector<int> M_;
    size_t idx(int l, int s) const { return (size_t)l * (S_ + 1) + s; }
};

}  // namespace semh
