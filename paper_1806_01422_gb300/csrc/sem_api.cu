// C ABI of libsem (declared in include/sem.h): handles, operator applies, the
// explicit Runge-Kutta forward sweep with trajectory storage, its discrete
// adjoint, the misfit, and one-call gradient evaluation.
//
// arXiv:1806.01422: the operators follow Sec. 3.3 (eqs. rhsvec, jacvec,
// jactransvec); the sweeps follow the adjoint derivation of Sec. 4.1 (eqs.
// adjointloop, initadj, gradient) carried through the stages of an explicit
// Butcher tableau; trajectory storage and recomputation follow Sec. 5.3-5.4.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include <algorithm>

#include "host_tables.h"
#include "sem.h"
#include "sem_internal.h"

using namespace semk;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define SEM_CK(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            cudaGetLastError(); /* a failed call must not be seen by the next launch check */ \
            return fail(SEM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));               \
        }                                                                                     \
    } while (0)

#define SEM_TRY(expr)                  \
    do {                               \
        int r_ = (expr);               \
        if (r_ != SEM_OK) return r_;   \
    } while (0)

// Explicit Butcher tableaux (A strictly lower triangular).
struct Tableau {
    int s;
    double A[4][4];
    double b[4];
};

// Stage i depends only on k_{i-1} (A is subdiagonal): RK4, forward Euler.  The
// sweeps then carry running sums instead of storing every stage derivative.
bool subdiagonal(const Tableau& t) {
    for (int i = 0; i < t.s; ++i)
        for (int j = 0; j + 1 < i; ++j)
            if (t.A[i][j] != 0.0) return false;
    return true;
}

bool tableau_of(int scheme, Tableau& t) {
    std::memset(&t, 0, sizeof(t));
    if (scheme == SEM_RK4) {
        t.s = 4;
        t.A[1][0] = 0.5;
        t.A[2][1] = 0.5;
        t.A[3][2] = 1.0;
        t.b[0] = 1.0 / 6.0; t.b[1] = 1.0 / 3.0; t.b[2] = 1.0 / 3.0; t.b[3] = 1.0 / 6.0;
        return true;
    }
    if (scheme == SEM_SSPRK3) {
        t.s = 3;
        t.A[1][0] = 1.0;
        t.A[2][0] = 0.25;
        t.A[2][1] = 0.25;
        t.b[0] = 1.0 / 6.0; t.b[1] = 1.0 / 6.0; t.b[2] = 2.0 / 3.0;
        return true;
    }
    if (scheme == SEM_EULER) {
        t.s = 1;
        t.b[0] = 1.0;
        return true;
    }
    if (scheme == SEM_BS3) {   // third-order member of the Bogacki-Shampine 3(2) pair
        t.s = 3;
        t.A[1][0] = 0.5;
        t.A[2][1] = 0.75;
        t.b[0] = 2.0 / 9.0; t.b[1] = 1.0 / 3.0; t.b[2] = 4.0 / 9.0;
        return true;
    }
    return false;
}

// Second-order companion weights of the pair on (k1, k2, k3, k4 = F(u_{n+1})).
constexpr double BS3_BHAT[4] = {7.0 / 24.0, 1.0 / 4.0, 1.0 / 3.0, 1.0 / 8.0};

}  // namespace

// Host state of a batch of independent 2D instances (sem_batch_create).
struct BatchHost {
    int count = 0;
    std::vector<BatchInst> inst;
    std::vector<unsigned char> mats;   // packed OpMats<double, NP> per instance
    std::vector<RowInfo> rows;
    std::vector<int> row_start;        // count + 1
    std::vector<double> J;             // per-instance misfit of the last evaluation
    // device copies (allocated on first use)
    BatchInst* d_inst = nullptr;
    unsigned char* d_mats = nullptr;
    RowInfo* d_rows = nullptr;
    int* d_row_start = nullptr;
    WorkItem* d_items = nullptr;
    int nitems = 0;
    double* d_J = nullptr;
    double* d_rowpart = nullptr;
    int threads = 0;                   // block size of the element kernel (autotuned)
    int blocks = 0;
    double tune_ms[8] = {0};
};

struct sem_ctx {
    BatchHost* batch = nullptr;
    int dim = 0, E = 0, N = 0, np = 0, G = 0;
    int precision = SEM_PREC_FP64, ckpt_mode = SEM_CKPT_AUTO, ckpt_slots = 0;
    int contraction = SEM_CONTRACT_CUDA_CORE;   // sem_set_contraction
    size_t ckpt_budget = 0;
    double nu = 0, L = 0, h = 0;
    std::vector<double> xi, w, Dh, mats, mw;
    size_t ndof = 0, lvec_elems = 0;
    int nelem = 0;
    // device workspaces
    void* lvec = nullptr;
    double* partials = nullptr;
    double* scal = nullptr;      // [0] objective
    unsigned* flag = nullptr;    // non-finite flag
    double* vecs = nullptr;      // NVEC state-sized work vectors
    double* frozen = nullptr;    // frozen advecting field a (a state; float pairs in the FP32 form) or null
    long long nlaunch = 0;       // element and assembly launches since the last forward sweep began
    double* traj = nullptr;
    size_t traj_vectors = 0;
    // last forward sweep
    bool have_fwd = false;
    int f_scheme = 0, f_nsteps = 0, f_mode = 0, f_slots = 0;
    double f_dt = 0;
    std::vector<int> f_ckpt;
    // adaptive stepping (SEM_BS3 with tolerances): settings, accepted steps of the last sweep
    double adapt_atol = 0.0, adapt_rtol = 0.0;
    std::vector<double> f_dts;
    long long f_rejected = 0;
    double* adapt_buf = nullptr;
    // two-level trajectory store: states [0, f_ndev) in HBM, [f_ndev, nsteps) in pinned host memory
    size_t host_budget = 0;
    double* host_traj = nullptr;
    size_t host_vectors = 0;
    int f_ndev = 0;
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_comp[3] = {}, ev_copy[3] = {}, ev_load[3] = {}, ev_done[3] = {};
    long long st[3] = {0, 0, 0};  // forward F applies, adjoint F applies, adjoint J^T applies
    // CUDA graph of one gradient evaluation (sem_set_graph), keyed on its arguments
    bool graph_on = false;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    struct GraphKey {
        int scheme, nsteps;
        double dt;
        const void *u0, *uo, *grad;
        bool operator==(const GraphKey& o) const {
            return scheme == o.scheme && nsteps == o.nsteps && dt == o.dt && u0 == o.u0 && uo == o.uo && grad == o.grad;
        }
    } graph_key{-1, 0, 0.0, nullptr, nullptr, nullptr};
    long long graph_replays = 0;
    int fixed_mode = -1, fixed_slots = 0;   // storage mode fixed before a graph recording
    // kernel timing inside a recorded graph: the sampled launches' event pairs are
    // nodes of the graph and are read after each replay
    bool capturing = false;
    std::vector<cudaEvent_t> gev_start, gev_stop;
    std::vector<int> gev_kind;
    std::vector<double> gev_bytes;
    // Crank-Nicolson: Newton / GMRES settings, Krylov workspace, counters
    double newton_rtol = 1e-12, krylov_rtol = 1e-12;
    int krylov_m = 30, krylov_maxit = 2000, newton_maxit = 30;
    double* kbasis = nullptr;     // krylov_m + 2 vectors: the basis and a work vector
    double* kpart = nullptr;      // multidot partials
    double* kscal = nullptr;      // device scalars (2 KMAX)
    long long cn_st[4] = {0, 0, 0, 0};  // Newton iterations, forward and adjoint Krylov steps, operator applies
    // opt-in kernel timing: event pairs per launch, drained when the pool fills
    int prof = 0;                 // 0: off; n: time one apply in n per kind
    long long prof_tick[4] = {0, 0, 0, 0};
    std::vector<cudaEvent_t> ev_start, ev_stop;
    std::vector<int> ev_kind;
    std::vector<double> ev_bytes;
    size_t ev_used = 0;
    double prof_ms[4] = {0, 0, 0, 0};
    long long prof_n[4] = {0, 0, 0, 0};
    double prof_bytes[4] = {0, 0, 0, 0};   // algorithmic bytes of the timed launches
};

namespace {

// work vector roles inside sem_ctx::vecs
// internal storage mode of a linear (frozen-advection) sweep: nothing stored
constexpr int MODE_LINEAR = 100;
// staging ring (device state slots) between the compute stream and host memory
constexpr int TWO_LEVEL_RING = 3;
// internal storage mode of an adaptive sweep: every accepted state, step sizes on the host
constexpr int MODE_ADAPTIVE = 101;

enum { V_K0 = 0, V_STAGE0 = 4, V_CUR0 = 7, V_CUR1 = 8, V_NU = 9, V_UN = 10, V_LAM = 11, NVEC = 12 };

// FP32 form: every sweep-internal state is a pair of FP32 planes (hi at [0, ndof),
// lo at [ndof, 2 ndof) floats), the same bytes as one double state.
bool f32(sem_t h) { return h->precision == SEM_PREC_FP32_BULK; }
float* fl(double* p) { return reinterpret_cast<float*>(p); }
const float* fl(const double* p) { return reinterpret_cast<const float*>(p); }

double* vec(sem_t h, int i) { return h->vecs + (size_t)i * h->ndof; }

bool overlap(const void* a, const void* b, size_t bytes) {
    if (!a || !b) return false;
    const char* pa = (const char*)a;
    const char* pb = (const char*)b;
    return pa < pb + bytes && pb < pa + bytes;
}

int check_state_ptr(const void* p, const char* name) {
    if (!p) return fail(SEM_ERR_ARG, "%s is null", name);
    if ((uintptr_t)p % 8) return fail(SEM_ERR_ARG, "%s is not 8-byte aligned", name);
    return SEM_OK;
}

int validate(const sem_opts* o) {
    if (!o) return fail(SEM_ERR_ARG, "opts is null");
    if (o->dim < 1 || o->dim > 3) return fail(SEM_ERR_ARG, "dim must be 1, 2 or 3 (got %d)", o->dim);
    if (o->E < 1) return fail(SEM_ERR_ARG, "E must be >= 1 (got %d)", o->E);
    if (o->N < 1 || o->N > 15) return fail(SEM_ERR_ARG, "N must be in [1, 15] (got %d)", o->N);
    if (!(o->nu >= 0.0) || !std::isfinite(o->nu)) return fail(SEM_ERR_ARG, "nu must be finite and >= 0");
    if (!std::isfinite(o->L)) return fail(SEM_ERR_ARG, "L must be finite");
    if (o->precision != SEM_PREC_FP64 && o->precision != SEM_PREC_FP32_BULK && o->precision != SEM_PREC_FP64_DF)
        return fail(SEM_ERR_ARG, "unknown precision %d", o->precision);
    if (o->ckpt_mode < SEM_CKPT_AUTO || o->ckpt_mode > SEM_CKPT_TWO_LEVEL)
        return fail(SEM_ERR_ARG, "unknown checkpoint mode %d", o->ckpt_mode);
    if (o->ckpt_mode == SEM_CKPT_BINOMIAL && o->ckpt_slots < 1)
        return fail(SEM_ERR_ARG, "binomial checkpointing needs ckpt_slots >= 1");
    const int np = o->N + 1;
    if (np > max_np(o->dim, o->precision == SEM_PREC_FP32_BULK))
        return fail(SEM_ERR_ARG, "order N=%d is not supported for dim=%d in this precision (max N=%d)", o->N,
                    o->dim, max_np(o->dim, o->precision == SEM_PREC_FP32_BULK) - 1);
    double G = (double)o->E * o->N, nd = o->dim;
    for (int d = 0; d < o->dim; ++d) nd *= G;
    if (nd > 2147483647.0) return fail(SEM_ERR_ARG, "problem too large: %.0f unknowns (max 2^31-1)", nd);
    double nl = 1.0;
    for (int d = 0; d < o->dim; ++d) nl *= (double)o->E * np;
    if (nl * o->dim > 4.0e9) return fail(SEM_ERR_ARG, "element-local buffer too large");
    return SEM_OK;
}

int ensure_workspace(sem_t h) {
    if (h->lvec) return SEM_OK;
    const size_t esz = h->precision == SEM_PREC_FP32_BULK ? sizeof(float) : sizeof(double);
    cudaError_t e;
    if ((e = cudaMalloc(&h->lvec, h->lvec_elems * esz)) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->partials, sizeof(double) * objective_blocks((unsigned)h->ndof))) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->scal, sizeof(double) * 4)) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->flag, sizeof(unsigned) * 4)) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->vecs, sizeof(double) * h->ndof * NVEC)) != cudaSuccess) {
        cudaFree(h->lvec); cudaFree(h->partials); cudaFree(h->scal); cudaFree(h->flag); cudaFree(h->vecs);
        h->lvec = nullptr; h->partials = nullptr; h->scal = nullptr; h->flag = nullptr; h->vecs = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SEM_ERR_OOM : SEM_ERR_CUDA, "workspace allocation: %s",
                    cudaGetErrorString(e));
    }
    return SEM_OK;
}

// ------------------------------------------------------------ kernel timing
constexpr size_t PROF_POOL = 4096;

int prof_drain(sem_t h) {
    if (h->ev_used == 0) return SEM_OK;
    SEM_CK(cudaEventSynchronize(h->ev_stop[h->ev_used - 1]));
    for (size_t i = 0; i < h->ev_used; ++i) {
        float ms = 0.f;
        SEM_CK(cudaEventElapsedTime(&ms, h->ev_start[i], h->ev_stop[i]));
        h->prof_ms[h->ev_kind[i]] += ms;
        h->prof_n[h->ev_kind[i]] += 1;
        h->prof_bytes[h->ev_kind[i]] += h->ev_bytes[i];
    }
    h->ev_used = 0;
    return SEM_OK;
}

// Returns the index of the event pair to record around one launch (-1: profiling off).
// bytes: the launch's algorithmic bytes, summed over the timed launches of its kind.
int prof_begin(sem_t h, int kind, cudaStream_t s, long long& slot, double bytes = 0.0) {
    slot = -1;
    if (!h->prof) return SEM_OK;
    if (h->prof_tick[kind]++ % h->prof != 0) return SEM_OK;
    if (h->capturing) {
        cudaEvent_t a, b;
        SEM_CK(cudaEventCreate(&a));
        SEM_CK(cudaEventCreate(&b));
        h->gev_start.push_back(a);
        h->gev_stop.push_back(b);
        h->gev_kind.push_back(kind);
        h->gev_bytes.push_back(bytes);
        slot = -2 - (long long)(h->gev_start.size() - 1);
        // an event recorded into a graph must be an external record node to be timed
        SEM_CK(cudaEventRecordWithFlags(a, s, cudaEventRecordExternal));
        return SEM_OK;
    }
    if (h->ev_start.empty()) {
        h->ev_start.resize(PROF_POOL);
        h->ev_stop.resize(PROF_POOL);
        h->ev_kind.resize(PROF_POOL);
        h->ev_bytes.resize(PROF_POOL);
        for (size_t i = 0; i < PROF_POOL; ++i) {
            SEM_CK(cudaEventCreate(&h->ev_start[i]));
            SEM_CK(cudaEventCreate(&h->ev_stop[i]));
        }
    }
    if (h->ev_used == PROF_POOL) SEM_TRY(prof_drain(h));
    slot = (long long)h->ev_used++;
    h->ev_kind[slot] = kind;
    h->ev_bytes[slot] = bytes;
    SEM_CK(cudaEventRecord(h->ev_start[slot], s));
    return SEM_OK;
}

int prof_end(sem_t h, long long slot, cudaStream_t s) {
    if (slot >= 0) SEM_CK(cudaEventRecord(h->ev_stop[slot], s));
    if (slot <= -2) SEM_CK(cudaEventRecordWithFlags(h->gev_stop[(size_t)(-2 - slot)], s, cudaEventRecordExternal));
    return SEM_OK;
}

// Accumulate the timed launches of the last graph replay (after its stream was synchronised).
int prof_graph_accumulate(sem_t h) {
    for (size_t i = 0; i < h->gev_start.size(); ++i) {
        float ms = 0.f;
        SEM_CK(cudaEventElapsedTime(&ms, h->gev_start[i], h->gev_stop[i]));
        h->prof_ms[h->gev_kind[i]] += ms;
        h->prof_n[h->gev_kind[i]] += 1;
        h->prof_bytes[h->gev_kind[i]] += h->gev_bytes[i];
    }
    return SEM_OK;
}

void prof_graph_release(sem_t h) {
    for (size_t i = 0; i < h->gev_start.size(); ++i) {
        cudaEventDestroy(h->gev_start[i]);
        cudaEventDestroy(h->gev_stop[i]);
    }
    h->gev_start.clear();
    h->gev_stop.clear();
    h->gev_kind.clear();
    h->gev_bytes.clear();
}

// Algorithmic bytes of one gather-scatter launch: the element-local values read
// once (FP32 in the FP32-bulk form, FP64 otherwise), every epilogue source read
// and every output written once, 8 bytes per unknown (FP64, or a float pair).
double asm_bytes(sem_t h, const Epi& ep) {
    const double lw = h->precision == SEM_PREC_FP32_BULK ? 4.0 : 8.0;
    return (double)h->lvec_elems * lw + (double)(ep.nout + ep.nsrc) * (double)h->ndof * 8.0;
}

// One operator apply: element kernel into the element-local buffer, then the
// gather-scatter sum with the given epilogue.  f2_in: the inputs are
// sweep-internal float-pair states (FP32 form), not caller doubles.
int batch_apply(sem_t h, int op, const double* u, const double* w, const Epi& ep, cudaStream_t s);

AsmArgs asm_args(sem_t h, int scale_mult) {
    AsmArgs aa;
    aa.D = h->dim;
    aa.E = h->E;
    aa.N = h->N;
    aa.G = h->G;
    aa.NP = h->np;
    aa.GD = (unsigned)(h->ndof / h->dim);
    aa.ndof = (unsigned)h->ndof;
    aa.scale_mult = scale_mult;
    return aa;
}

// One operator apply: element kernel, then the gather-scatter with the epilogue `ep`.
int apply(sem_t h, int op, const double* u, const double* w, const Epi& ep, cudaStream_t s, bool f2_in = false) {
    if (h->batch) return batch_apply(h, op, u, w, ep, s);
    ElemArgs a;
    std::memset(&a, 0, sizeof(a));
    a.u = u;
    a.w = w;
    a.plane = (unsigned)h->ndof;
    a.in_f2 = f2_in ? 1 : 0;
    a.lvec = h->lvec;
    a.E = h->E;
    a.N = h->N;
    a.G = h->G;
    a.nelem = h->nelem;
    const bool f32 = h->precision == SEM_PREC_FP32_BULK;
    long long slot;
    SEM_TRY(prof_begin(h, op, s, slot));
    cudaError_t e;
    const double* mt = h->mats.data();
    if (h->contraction == SEM_CONTRACT_TENSOR && tc_supported(h->dim, h->np, op, f32)) {
        e = launch_elem_tc(f32, op, mt, a, h->flag ? h->flag + 1 : nullptr, s);
    } else if (h->precision == SEM_PREC_FP64_DF) {   // double-float element arithmetic, FP64 everywhere else
        if (h->dim == 1) e = launch_elem<dfloat, 1>(h->np, op, mt, a, s);
        else if (h->dim == 2) e = launch_elem<dfloat, 2>(h->np, op, mt, a, s);
        else e = launch_elem<dfloat, 3>(h->np, op, mt, a, s);
    } else if (h->dim == 1) {
        e = f32 ? launch_elem<float, 1>(h->np, op, mt, a, s) : launch_elem<double, 1>(h->np, op, mt, a, s);
    } else if (h->dim == 2) {
        e = f32 ? launch_elem<float, 2>(h->np, op, mt, a, s) : launch_elem<double, 2>(h->np, op, mt, a, s);
    } else {
        e = f32 ? launch_elem<float, 3>(h->np, op, mt, a, s) : launch_elem<double, 3>(h->np, op, mt, a, s);
    }
    if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "element kernel launch: %s", cudaGetErrorString(e));
    SEM_TRY(prof_end(h, slot, s));
    ++h->nlaunch;
    SEM_TRY(prof_begin(h, 3, s, slot, asm_bytes(h, ep)));
    e = launch_assemble(f32, a.lvec, asm_args(h, op != OP_JACT), ep, s);
    if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "assembly launch: %s", cudaGetErrorString(e));
    SEM_TRY(prof_end(h, slot, s));
    ++h->nlaunch;
    return SEM_OK;
}

Epi epi_plain(double* out, unsigned* flag) {
    Epi ep;
    std::memset(&ep, 0, sizeof(ep));
    ep.out[0] = out;
    ep.alpha[0] = 1.0;
    ep.nout = 1;
    ep.nonfinite = flag;
    return ep;
}

int add_src(Epi& ep, const double* p) {
    for (int m = 0; m < ep.nsrc; ++m)
        if (ep.src[m] == p) return m;
    ep.src[ep.nsrc] = p;
    return ep.nsrc++;
}

// Forward stages of one step from un (Sec. 4.1 model u_{n+1} = A(u_n, P[u_n])):
//   Y_1 = un, Y_{i+1} = un + dt sum_{j<=i} A[i+1][j] k_j,  k_i = F(Y_i).
// Y_{i+1} goes to Y[i+1] (Y[0] is un); k_i to vec(V_K0 + i).  If unext is
// non-null the last stage writes u_{n+1} = un + dt sum_i b_i k_i; otherwise the
// step stops after Y_s (taping only: s-1 applies).
// The stage derivative k = F(Y), or J(a) Y with a frozen advecting field a.
int stage_rhs(sem_t h, const double* Y, const Epi& ep, cudaStream_t s) {
    if (h->frozen) return apply(h, OP_JAC, h->frozen, Y, ep, s, f32(h));
    return apply(h, OP_RHS, Y, nullptr, ep, s, f32(h));
}

// The linearisation point of the adjoint stage: Y itself, or the frozen field.
const double* jac_point(sem_t h, const double* Y) { return h->frozen ? h->frozen : Y; }

int rk_stages(sem_t h, const Tableau& T, double dt, const double* un, double* const* Y, double* unext,
              cudaStream_t s, long long& count) {
    const int last = unext ? T.s - 1 : T.s - 2;
    if (subdiagonal(T)) {
        // Y_{i+1} = un + dt a_{i+1,i} k_i and the running sum acc = un + dt sum_{j<=i} b_j k_j
        // (vec(V_K0)); the last stage writes unext = acc + dt b_{s-1} k_{s-1}.
        double* acc = vec(h, V_K0);
        for (int i = 0; i <= last; ++i) {
            Epi ep;
            std::memset(&ep, 0, sizeof(ep));
            ep.nonfinite = h->flag;
            ep.f2 = f32(h);
            if (i < T.s - 1) {
                const int su = add_src(ep, un);
                ep.out[0] = Y[i + 1];
                ep.alpha[0] = dt * T.A[i + 1][i];
                ep.beta[0][su] = 1.0;
                ep.nout = 1;
                if (unext) {
                    const int sa = i == 0 ? su : add_src(ep, acc);
                    ep.out[1] = acc;
                    ep.alpha[1] = dt * T.b[i];
                    ep.beta[1][sa] = 1.0;
                    ep.nout = 2;
                }
            } else {
                const int sa = T.s == 1 ? add_src(ep, un) : add_src(ep, acc);
                ep.out[0] = unext;
                ep.alpha[0] = dt * T.b[i];
                ep.beta[0][sa] = 1.0;
                ep.nout = 1;
            }
            SEM_TRY(stage_rhs(h, i == 0 ? un : Y[i], ep, s));
            ++count;
        }
        return SEM_OK;
    }
    for (int i = 0; i <= last; ++i) {
        const double* Yi = i == 0 ? un : Y[i];
        Epi ep;
        std::memset(&ep, 0, sizeof(ep));
        ep.nonfinite = h->flag;
        ep.f2 = f32(h);
        const int su = add_src(ep, un);
        if (i < T.s - 1) {
            ep.out[0] = Y[i + 1];
            ep.alpha[0] = dt * T.A[i + 1][i];
            ep.beta[0][su] = 1.0;
            for (int j = 0; j < i; ++j)
                if (T.A[i + 1][j] != 0.0) ep.beta[0][add_src(ep, vec(h, V_K0 + j))] = dt * T.A[i + 1][j];
            ep.out[1] = vec(h, V_K0 + i);
            ep.alpha[1] = 1.0;
            ep.nout = 2;
        } else {
            ep.out[0] = unext;
            ep.alpha[0] = dt * T.b[i];
            ep.beta[0][su] = 1.0;
            for (int j = 0; j < i; ++j)
                if (T.b[j] != 0.0) ep.beta[0][add_src(ep, vec(h, V_K0 + j))] = dt * T.b[j];
            ep.nout = 1;
        }
        SEM_TRY(stage_rhs(h, Yi, ep, s));
        ++count;
    }
    return SEM_OK;
}

// Discrete adjoint of one step given its stage values Y[0..s-1] (Sec. 4.1):
//   for i = s-1..0:  mu_i = J(Y_i)^T nu_i,
//                    nu_{i-1} = dt (b_{i-1} lam + sum_{j > i-1} A[j][i-1] mu_j),
//   lam <- lam + sum_i mu_i.
// On entry vec(V_NU) holds nu_{s-1} = dt b_{s-1} lam; on exit it holds the same
// quantity for the updated lam (the next step's first stage).  lam is updated in place.
int rk_adjoint_step(sem_t h, const Tableau& T, double dt, const double* const* Y, double* lam,
                    cudaStream_t s, long long& count, double dt_next = -1.0) {
    if (dt_next < 0) dt_next = dt;   // step size of the next (earlier) step, for its nu_{s-1}
    double* nu = vec(h, V_NU);
    if (subdiagonal(T) && T.s > 1) {
        // nu_{i-1} = dt (b_{i-1} lam + a_{i,i-1} mu_i) and the running sum
        // lacc = lam + sum_{j>=i} mu_j (vec(V_K0)); stage 0 writes lam = lacc + mu_0 and
        // the next step's nu_{s-1} = dt b_{s-1} lam.
        double* lacc = vec(h, V_K0);
        for (int i = T.s - 1; i >= 0; --i) {
            Epi ep;
            std::memset(&ep, 0, sizeof(ep));
            ep.nonfinite = h->flag;
            ep.f2 = f32(h);
            if (i > 0) {
                const int sl = add_src(ep, lam);
                ep.out[0] = nu;
                ep.alpha[0] = dt * T.A[i][i - 1];
                ep.beta[0][sl] = dt * T.b[i - 1];
                const int sa = i == T.s - 1 ? sl : add_src(ep, lacc);
                ep.out[1] = lacc;
                ep.alpha[1] = 1.0;
                ep.beta[1][sa] = 1.0;
                ep.nout = 2;
            } else {
                const int sa = add_src(ep, lacc);
                ep.out[0] = lam;
                ep.alpha[0] = 1.0;
                ep.beta[0][sa] = 1.0;
                const double c = dt_next * T.b[T.s - 1];
                ep.out[1] = nu;
                ep.alpha[1] = c;
                ep.beta[1][sa] = c;
                ep.nout = 2;
            }
            SEM_TRY(apply(h, OP_JACT, jac_point(h, Y[i]), nu, ep, s, f32(h)));
            ++count;
        }
        return SEM_OK;
    }
    for (int i = T.s - 1; i >= 0; --i) {
        Epi ep;
        std::memset(&ep, 0, sizeof(ep));
        ep.nonfinite = h->flag;
        ep.f2 = f32(h);
        const int sl = add_src(ep, lam);
        if (i > 0) {
            ep.out[0] = nu;
            ep.alpha[0] = dt * T.A[i][i - 1];
            ep.beta[0][sl] = dt * T.b[i - 1];
            for (int j = i + 1; j < T.s; ++j)
                if (T.A[j][i - 1] != 0.0) ep.beta[0][add_src(ep, vec(h, V_K0 + j))] = dt * T.A[j][i - 1];
            ep.out[1] = vec(h, V_K0 + i);
            ep.alpha[1] = 1.0;
            ep.nout = 2;
        } else {
            ep.out[0] = lam;
            ep.alpha[0] = 1.0;
            ep.beta[0][sl] = 1.0;
            for (int j = 1; j < T.s; ++j) ep.beta[0][add_src(ep, vec(h, V_K0 + j))] = 1.0;
            const double c = dt_next * T.b[T.s - 1];
            ep.out[1] = nu;
            ep.alpha[1] = c;
            for (int m = 0; m < ep.nsrc; ++m) ep.beta[1][m] = c * ep.beta[0][m];
            ep.nout = 2;
        }
        SEM_TRY(apply(h, OP_JACT, jac_point(h, Y[i]), nu, ep, s, f32(h)));
        ++count;
    }
    return SEM_OK;
}

size_t vec_bytes(sem_t h) { return h->ndof * sizeof(double); }

int alloc_traj(sem_t h, size_t nvec) {
    if (h->traj && h->traj_vectors >= nvec) return SEM_OK;
    if (h->traj) {
        cudaFree(h->traj);
        h->traj = nullptr;
        h->traj_vectors = 0;
    }
    if (h->ckpt_budget && nvec * vec_bytes(h) > h->ckpt_budget)
        return fail(SEM_ERR_OOM, "trajectory needs %zu bytes, budget is %zu", nvec * vec_bytes(h), h->ckpt_budget);
    cudaError_t e = cudaMalloc((void**)&h->traj, nvec * vec_bytes(h));
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->traj = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? SEM_ERR_OOM : SEM_ERR_CUDA,
                    "trajectory allocation of %zu bytes: %s", nvec * vec_bytes(h), cudaGetErrorString(e));
    }
    h->traj_vectors = nvec;
    return SEM_OK;
}

// Device budget of the trajectory (explicit, or free memory less 4 GiB of headroom).
size_t device_budget(sem_t h) {
    if (h->ckpt_budget) return h->ckpt_budget;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        fr = 0;
    }
    fr += h->traj ? h->traj_vectors * vec_bytes(h) : 0;
    const size_t headroom = (size_t)4 << 30;
    return fr > headroom ? fr - headroom : fr / 2;
}

// Storage mode for a sweep of nsteps steps of an s-stage scheme.
int choose_mode(sem_t h, int s, int nsteps, int& mode, int& slots) {
    if (h->fixed_mode >= 0) {
        mode = h->fixed_mode;
        slots = h->fixed_slots;
        return SEM_OK;
    }
    mode = h->ckpt_mode;
    slots = h->ckpt_slots;
    if (mode != SEM_CKPT_AUTO) return SEM_OK;
    // without an explicit budget: the free device memory (plus the trajectory buffer
    // this handle would release) minus 4 GiB of headroom for other users
    const size_t budget = device_budget(h);
    const size_t v = vec_bytes(h);
    if ((size_t)nsteps * s * v <= budget) mode = SEM_CKPT_STAGES;
    else if ((size_t)nsteps * v <= budget) mode = SEM_CKPT_STATES;
    else if (h->host_budget && budget >= TWO_LEVEL_RING * v &&
             (size_t)nsteps * v <= budget - TWO_LEVEL_RING * v + h->host_budget)
        mode = SEM_CKPT_TWO_LEVEL;
    else {
        mode = SEM_CKPT_BINOMIAL;
        slots = (int)(budget / v);
        if (slots < 1) return fail(SEM_ERR_OOM, "not even one checkpoint slot fits in %zu bytes", budget);
    }
    return SEM_OK;
}

// Two-level store: the copy stream, its events and the pinned host buffer for nhost states.
int two_level_setup(sem_t h, size_t nhost) {
    if (!h->cstream) SEM_CK(cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking));
    for (int k = 0; k < TWO_LEVEL_RING; ++k) {
        if (!h->ev_comp[k]) SEM_CK(cudaEventCreateWithFlags(&h->ev_comp[k], cudaEventDisableTiming));
        if (!h->ev_copy[k]) SEM_CK(cudaEventCreateWithFlags(&h->ev_copy[k], cudaEventDisableTiming));
        if (!h->ev_load[k]) SEM_CK(cudaEventCreateWithFlags(&h->ev_load[k], cudaEventDisableTiming));
        if (!h->ev_done[k]) SEM_CK(cudaEventCreateWithFlags(&h->ev_done[k], cudaEventDisableTiming));
    }
    if (nhost * vec_bytes(h) > h->host_budget)
        return fail(SEM_ERR_OOM, "%zu host states exceed the host budget of %zu bytes", nhost, h->host_budget);
    if (h->host_traj && h->host_vectors >= nhost) return SEM_OK;
    if (h->host_traj) {
        SEM_CK(cudaStreamSynchronize(h->cstream));
        cudaFreeHost(h->host_traj);
        h->host_traj = nullptr;
        h->host_vectors = 0;
    }
    cudaError_t e = cudaMallocHost((void**)&h->host_traj, nhost * vec_bytes(h));
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->host_traj = nullptr;
        return fail(SEM_ERR_OOM, "pinned host trajectory of %zu bytes: %s", nhost * vec_bytes(h),
                    cudaGetErrorString(e));
    }
    h->host_vectors = nhost;
    return SEM_OK;
}

int check_flag(sem_t h, cudaStream_t s, const char* what) {
    unsigned f = 0;
    SEM_CK(cudaMemcpyAsync(&f, h->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SEM_CK(cudaStreamSynchronize(s));
    if (f) return fail(SEM_ERR_NONFINITE, "non-finite values in the %s sweep", what);
    return SEM_OK;
}

int cn_forward(sem_t h, double dt, int nsteps, const double* u0, double* uT, cudaStream_t s);
int cn_adjoint(sem_t h, const double* lamT, double* lam0, cudaStream_t s);
int adaptive_forward(sem_t h, double T, double dt0, const double* u0, double* uT, cudaStream_t s);
bool adaptive(sem_t h, int scheme) { return scheme == SEM_BS3 && (h->adapt_atol > 0.0 || h->adapt_rtol > 0.0); }

// uT_internal: uT is a handle work state (float pairs in the FP32 form) rather
// than the caller's double output.
int forward_impl(sem_t h, int scheme, double dt, int nsteps, const double* u0, double* uT, cudaStream_t s,
                 bool uT_internal = false) {
    Tableau T;
    if (scheme != SEM_CN && !tableau_of(scheme, T)) return fail(SEM_ERR_ARG, "unknown time scheme %d", scheme);
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(SEM_ERR_ARG, "dt must be finite and > 0");
    if (nsteps < 1) return fail(SEM_ERR_ARG, "nsteps must be >= 1");
    SEM_TRY(check_state_ptr(u0, "u0"));
    SEM_TRY(check_state_ptr(uT, "uT"));
    if (overlap(u0, uT, vec_bytes(h))) return fail(SEM_ERR_ALIAS, "uT overlaps u0");
    SEM_TRY(ensure_workspace(h));
    h->nlaunch = 0;
    if (scheme == SEM_CN) return cn_forward(h, dt, nsteps, u0, uT, s);
    if (adaptive(h, scheme)) return adaptive_forward(h, dt * nsteps, dt, u0, uT, s);
    int mode, slots;
    SEM_TRY(choose_mode(h, T.s, nsteps, mode, slots));
    if (mode == SEM_CKPT_BINOMIAL && slots > nsteps) slots = nsteps;
    if (h->frozen) mode = MODE_LINEAR;   // the adjoint needs no stage values
    int ndev = nsteps;
    if (mode == SEM_CKPT_TWO_LEVEL) {
        if (!h->host_budget) return fail(SEM_ERR_ARG, "two-level storage needs a host budget (sem_set_host_tier)");
        const size_t fit = device_budget(h) / vec_bytes(h);
        if (fit < (size_t)TWO_LEVEL_RING) return fail(SEM_ERR_OOM, "the device budget holds fewer than 3 states");
        ndev = (int)std::min<size_t>((size_t)nsteps, fit - TWO_LEVEL_RING);
        SEM_TRY(two_level_setup(h, (size_t)(nsteps - ndev)));
    }
    const size_t nvec = mode == SEM_CKPT_STAGES ? (size_t)nsteps * T.s
                        : mode == SEM_CKPT_STATES ? (size_t)nsteps
                        : mode == SEM_CKPT_TWO_LEVEL ? (size_t)ndev + TWO_LEVEL_RING : (size_t)slots;
    if (mode != MODE_LINEAR) SEM_TRY(alloc_traj(h, nvec));
    h->have_fwd = false;
    const size_t vb = vec_bytes(h);
    double* Yw[4] = {nullptr, vec(h, V_STAGE0), vec(h, V_STAGE0 + 1), vec(h, V_STAGE0 + 2)};
    long long count = 0;
    std::vector<int> ckpt;
    // the final state: in the FP32 form it is produced as float pairs and widened at the end
    double* const uT_caller = uT;
    const bool widen_out = f32(h) && !uT_internal;
    if (widen_out) uT = vec(h, V_UN);
    auto put_u0 = [&](double* dst) -> int {
        if (f32(h)) {
            cudaError_t e = launch_f64_to_f2(u0, fl(dst), h->ndof, s);
            if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "conversion launch: %s", cudaGetErrorString(e));
        } else {
            SEM_CK(cudaMemcpyAsync(dst, u0, vb, cudaMemcpyDeviceToDevice, s));
        }
        return SEM_OK;
    };
    if (mode == MODE_LINEAR) {
        SEM_TRY(put_u0(vec(h, V_CUR0)));
        const double* cur = vec(h, V_CUR0);
        for (int n = 0; n < nsteps; ++n) {
            double* next = n + 1 == nsteps ? uT : (cur == vec(h, V_CUR0) ? vec(h, V_CUR1) : vec(h, V_CUR0));
            SEM_TRY(rk_stages(h, T, dt, cur, Yw, next, s, count));
            cur = next;
        }
    } else if (mode == SEM_CKPT_STAGES) {
        SEM_TRY(put_u0(h->traj));
        for (int n = 0; n < nsteps; ++n) {
            double* base = h->traj + (size_t)n * T.s * h->ndof;
            double* Y[4] = {base, base + h->ndof, base + 2 * h->ndof, base + 3 * h->ndof};
            double* next = n + 1 < nsteps ? h->traj + (size_t)(n + 1) * T.s * h->ndof : uT;
            SEM_TRY(rk_stages(h, T, dt, base, Y, next, s, count));
        }
    } else if (mode == SEM_CKPT_STATES) {
        SEM_TRY(put_u0(h->traj));
        for (int n = 0; n < nsteps; ++n) {
            const double* un = h->traj + (size_t)n * h->ndof;
            double* next = n + 1 < nsteps ? h->traj + (size_t)(n + 1) * h->ndof : uT;
            SEM_TRY(rk_stages(h, T, dt, un, Yw, next, s, count));
        }
    } else if (mode == SEM_CKPT_TWO_LEVEL) {
        // states n < ndev in HBM; later ones through the staging ring to pinned host memory,
        // copied on the copy stream while the next steps compute
        auto slot = [&](int n) -> double* {
            return h->traj + (size_t)(n < ndev ? n : ndev + n % TWO_LEVEL_RING) * h->ndof;
        };
        bool pending[TWO_LEVEL_RING] = {false, false, false};
        auto offload = [&](int n) -> int {
            const int k = n % TWO_LEVEL_RING;
            SEM_CK(cudaEventRecord(h->ev_comp[k], s));
            SEM_CK(cudaStreamWaitEvent(h->cstream, h->ev_comp[k], 0));
            SEM_CK(cudaMemcpyAsync(h->host_traj + (size_t)(n - ndev) * h->ndof, slot(n), vb, cudaMemcpyDeviceToHost,
                                   h->cstream));
            SEM_CK(cudaEventRecord(h->ev_copy[k], h->cstream));
            pending[k] = true;
            return SEM_OK;
        };
        auto claim = [&](int n) -> int {   // the ring slot of state n may be overwritten
            const int k = n % TWO_LEVEL_RING;
            if (pending[k]) SEM_CK(cudaStreamWaitEvent(s, h->ev_copy[k], 0));
            pending[k] = false;
            return SEM_OK;
        };
        if (ndev == 0) SEM_TRY(claim(0));
        SEM_TRY(put_u0(slot(0)));
        if (ndev == 0) SEM_TRY(offload(0));
        for (int n = 0; n < nsteps; ++n) {
            const bool last = n + 1 == nsteps;
            const bool to_host = !last && n + 1 >= ndev;
            if (to_host) SEM_TRY(claim(n + 1));
            SEM_TRY(rk_stages(h, T, dt, slot(n), Yw, last ? uT : slot(n + 1), s, count));
            if (to_host) SEM_TRY(offload(n + 1));
        }
        for (int k = 0; k < TWO_LEVEL_RING; ++k)
            if (pending[k]) SEM_CK(cudaStreamWaitEvent(s, h->ev_copy[k], 0));
    } else {
        semh::CkptPlanner P(nsteps, slots);
        ckpt = P.forward_checkpoints(nsteps, slots);
        SEM_TRY(put_u0(h->traj));
        const double* cur = h->traj;
        size_t k = 1;
        for (int n = 0; n < nsteps; ++n) {
            double* next;
            if (n + 1 == nsteps) next = uT;
            else if (k < ckpt.size() && ckpt[k] == n + 1) next = h->traj + (size_t)(k++) * h->ndof;
            else next = cur == vec(h, V_CUR0) ? vec(h, V_CUR1) : vec(h, V_CUR0);
            SEM_TRY(rk_stages(h, T, dt, cur, Yw, next, s, count));
            cur = next;
        }
    }
    if (widen_out) {
        cudaError_t e = launch_f2_to_f64(fl(uT), uT_caller, h->ndof, s);
        if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "conversion launch: %s", cudaGetErrorString(e));
    }
    h->have_fwd = true;
    h->f_scheme = scheme;
    h->f_nsteps = nsteps;
    h->f_dt = dt;
    h->f_mode = mode;
    h->f_slots = slots;
    h->f_ckpt = ckpt;
    h->f_ndev = mode == SEM_CKPT_TWO_LEVEL ? ndev : 0;
    h->st[0] = count;
    return SEM_OK;
}

// lam_internal (FP32 form only): the terminal adjoint is already in vec(V_LAM).
int adjoint_impl(sem_t h, const double* lamT, double* lam0, cudaStream_t s, bool lam_internal = false) {
    if (!h->have_fwd) return fail(SEM_ERR_STATE, "sem_rk_adjoint needs a completed sem_rk_forward");
    if (!lam_internal) SEM_TRY(check_state_ptr(lamT, "lamT"));
    SEM_TRY(check_state_ptr(lam0, "lam0"));
    if (lamT != lam0 && overlap(lamT, lam0, vec_bytes(h))) return fail(SEM_ERR_ALIAS, "lam0 partially overlaps lamT");
    if (h->f_scheme == SEM_CN) return cn_adjoint(h, lamT, lam0, s);
    Tableau T;
    tableau_of(h->f_scheme, T);
    const double dt = h->f_dt;
    const int nsteps = h->f_nsteps;
    const size_t vb = vec_bytes(h);
    double* const lam_out = lam0;
    if (f32(h)) {
        // the adjoint runs on float pairs in vec(V_LAM); lam0 is written at the end
        lam0 = vec(h, V_LAM);
        if (!lam_internal) {
            cudaError_t e = launch_f64_to_f2(lamT, fl(lam0), h->ndof, s);
            if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "conversion launch: %s", cudaGetErrorString(e));
        }
        cudaError_t e = launch_scale_f2(fl(vec(h, V_NU)), fl(lam0), dt * T.b[T.s - 1], h->ndof, s);
        if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "scale launch: %s", cudaGetErrorString(e));
    } else {
        if (lam0 != lamT) SEM_CK(cudaMemcpyAsync(lam0, lamT, vb, cudaMemcpyDeviceToDevice, s));
        cudaError_t e = launch_scale(vec(h, V_NU), lam0, dt * T.b[T.s - 1], h->ndof, s);
        if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "scale launch: %s", cudaGetErrorString(e));
    }
    long long nrhs = 0, njt = 0;
    double* Yw[4] = {nullptr, vec(h, V_STAGE0), vec(h, V_STAGE0 + 1), vec(h, V_STAGE0 + 2)};
    if (h->f_mode == MODE_ADAPTIVE) {
        // accepted steps in reverse, each with its own step size; stages recomputed from its state
        for (int n = nsteps - 1; n >= 0; --n) {
            double* un = h->traj + (size_t)n * h->ndof;
            Yw[0] = un;
            SEM_TRY(rk_stages(h, T, h->f_dts[n], un, Yw, nullptr, s, nrhs));
            const double* Y[4] = {Yw[0], Yw[1], Yw[2], Yw[3]};
            SEM_TRY(rk_adjoint_step(h, T, h->f_dts[n], Y, lam0, s, njt, n > 0 ? h->f_dts[n - 1] : h->f_dts[n]));
        }
    } else if (h->f_mode == MODE_LINEAR) {
        if (!h->frozen) return fail(SEM_ERR_STATE, "the advecting field changed after the forward sweep");
        const double* Y[4] = {h->frozen, h->frozen, h->frozen, h->frozen};
        for (int n = nsteps - 1; n >= 0; --n) SEM_TRY(rk_adjoint_step(h, T, dt, Y, lam0, s, njt));
    } else if (h->f_mode == SEM_CKPT_STAGES) {
        for (int n = nsteps - 1; n >= 0; --n) {
            double* base = h->traj + (size_t)n * T.s * h->ndof;
            const double* Y[4] = {base, base + h->ndof, base + 2 * h->ndof, base + 3 * h->ndof};
            SEM_TRY(rk_adjoint_step(h, T, dt, Y, lam0, s, njt));
        }
    } else if (h->f_mode == SEM_CKPT_STATES) {
        for (int n = nsteps - 1; n >= 0; --n) {
            double* un = h->traj + (size_t)n * h->ndof;
            Yw[0] = un;
            SEM_TRY(rk_stages(h, T, dt, un, Yw, nullptr, s, nrhs));
            const double* Y[4] = {Yw[0], Yw[1], Yw[2], Yw[3]};
            SEM_TRY(rk_adjoint_step(h, T, dt, Y, lam0, s, njt));
        }
    } else if (h->f_mode == SEM_CKPT_TWO_LEVEL) {
        // host states come back through the staging ring, loaded up to 3 steps ahead on the copy stream
        const int ndev = h->f_ndev;
        bool used[TWO_LEVEL_RING] = {false, false, false};
        // the copy stream starts after everything the caller queued before this sweep on s
        SEM_CK(cudaEventRecord(h->ev_comp[0], s));
        SEM_CK(cudaStreamWaitEvent(h->cstream, h->ev_comp[0], 0));
        auto ring = [&](int n) { return h->traj + (size_t)(ndev + n % TWO_LEVEL_RING) * h->ndof; };
        auto load = [&](int n) -> int {
            const int k = n % TWO_LEVEL_RING;
            if (used[k]) SEM_CK(cudaStreamWaitEvent(h->cstream, h->ev_done[k], 0));
            SEM_CK(cudaMemcpyAsync(ring(n), h->host_traj + (size_t)(n - ndev) * h->ndof, vb, cudaMemcpyHostToDevice,
                                   h->cstream));
            SEM_CK(cudaEventRecord(h->ev_load[k], h->cstream));
            return SEM_OK;
        };
        for (int n = nsteps - 1; n >= std::max(ndev, nsteps - TWO_LEVEL_RING); --n) SEM_TRY(load(n));
        for (int n = nsteps - 1; n >= 0; --n) {
            const bool host = n >= ndev;
            double* un = host ? ring(n) : h->traj + (size_t)n * h->ndof;
            if (host) SEM_CK(cudaStreamWaitEvent(s, h->ev_load[n % TWO_LEVEL_RING], 0));
            Yw[0] = un;
            SEM_TRY(rk_stages(h, T, dt, un, Yw, nullptr, s, nrhs));
            const double* Y[4] = {Yw[0], Yw[1], Yw[2], Yw[3]};
            SEM_TRY(rk_adjoint_step(h, T, dt, Y, lam0, s, njt));   // reads u_n as stage 0
            if (host) {
                SEM_CK(cudaEventRecord(h->ev_done[n % TWO_LEVEL_RING], s));
                used[n % TWO_LEVEL_RING] = true;
                if (n - TWO_LEVEL_RING >= ndev) SEM_TRY(load(n - TWO_LEVEL_RING));
            }
        }
    } else {
        semh::CkptPlanner P(nsteps, h->f_slots);
        const std::vector<semh::CkptAction> acts = P.backward_actions(nsteps, h->f_slots);
        const double* cur = nullptr;
        for (const semh::CkptAction& a : acts) {
            if (a.kind == semh::CkptAction::RESTORE) {
                cur = h->traj + (size_t)a.arg * h->ndof;
            } else if (a.kind == semh::CkptAction::ADVANCE) {
                for (int k = 0; k < a.arg; ++k) {
                    double* next = cur == vec(h, V_CUR0) ? vec(h, V_CUR1) : vec(h, V_CUR0);
                    SEM_TRY(rk_stages(h, T, dt, cur, Yw, next, s, nrhs));
                    cur = next;
                }
            } else if (a.kind == semh::CkptAction::STORE) {
                SEM_CK(cudaMemcpyAsync(h->traj + (size_t)a.arg * h->ndof, cur, vb, cudaMemcpyDeviceToDevice, s));
            } else {
                Yw[0] = const_cast<double*>(cur);
                SEM_TRY(rk_stages(h, T, dt, cur, Yw, nullptr, s, nrhs));
                const double* Y[4] = {Yw[0], Yw[1], Yw[2], Yw[3]};
                SEM_TRY(rk_adjoint_step(h, T, dt, Y, lam0, s, njt));
            }
        }
    }
    if (f32(h)) {
        cudaError_t e = launch_f2_to_f64(fl(lam0), lam_out, h->ndof, s);
        if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "conversion launch: %s", cudaGetErrorString(e));
    }
    h->st[1] = nrhs;
    h->st[2] = njt;
    return SEM_OK;
}

// f2_state (FP32 form): u and lam are float-pair work states.
int batch_objective(sem_t h, const double* u, const double* uo, double* lam, cudaStream_t s);

int objective_impl(sem_t h, const double* u, const double* uo, double* lam, cudaStream_t s, bool f2_state = false) {
    if (h->batch) return batch_objective(h, u, uo, lam, s);
    ObjArgs a;
    std::memset(&a, 0, sizeof(a));
    a.D = h->dim;
    a.N = h->N;
    a.G = h->G;
    a.GD = (unsigned)(h->ndof / h->dim);
    a.ndof = (unsigned)h->ndof;
    for (int i = 0; i < h->N; ++i) a.mw[i] = h->mw[i];
    a.scale = std::pow(h->h / 2.0, h->dim);
    const int nb = objective_blocks(a.ndof);
    cudaError_t e = f2_state ? launch_objective_f2(fl(u), uo, fl(lam), h->partials, nb, a, s)
                             : launch_objective(u, uo, lam, h->partials, nb, a, s);
    if (e == cudaSuccess) e = launch_sum_partials(h->partials, nb, h->scal, 0.5, s);
    if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "objective launch: %s", cudaGetErrorString(e));
    return SEM_OK;
}

// ------------------------------------------------------------------ Crank-Nicolson
// The implicit scheme of Sec. 6.3.  Step: R(v) = v - u_n - dt/2 (F(u_n) + F(v)) = 0
// by Newton, (I - dt/2 J(v)) delta = -R(v), each linear system by restarted GMRES;
// discrete adjoint: (I - dt/2 J(u_{n+1})^T) mu = lam_{n+1}, lam_n = mu + dt/2 J(u_n)^T mu.
// The Newton right-hand side and the products (I - c J) x are operator applies
// whose assembly epilogue adds the shifts, so every step runs in the library's
// kernels.  GMRES keeps its basis on the device (classical Gram-Schmidt with one
// re-orthogonalisation, coefficients never leave the device) and reads back the
// new Hessenberg column once per Arnoldi step for the Givens rotations.
constexpr int KSCAL_ONE = 2 * KMAX;   // kscal[KSCAL_ONE] == 1.0

int krylov_ws(sem_t h) {
    if (h->kbasis) return SEM_OK;
    cudaError_t e = cudaMalloc((void**)&h->kbasis, vec_bytes(h) * (h->krylov_m + 2));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->kpart, sizeof(double) * KMAX * multidot_blocks(h->ndof));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->kscal, sizeof(double) * (KSCAL_ONE + 1));
    if (e == cudaSuccess) {
        const double one = 1.0;
        e = cudaMemcpy(h->kscal + KSCAL_ONE, &one, sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->kbasis);
        cudaFree(h->kpart);
        cudaFree(h->kscal);
        h->kbasis = nullptr;
        h->kpart = h->kscal = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? SEM_ERR_OOM : SEM_ERR_CUDA, "Krylov workspace: %s",
                    cudaGetErrorString(e));
    }
    return SEM_OK;
}

double* kvec(sem_t h, int j) { return h->kbasis + (size_t)j * h->ndof; }

// device scalars out[0..k) = <V_j, w>
int dots(sem_t h, const double* const* V, int k, const double* w, double* out, cudaStream_t s) {
    VecList L;
    for (int j = 0; j < k; ++j) L.v[j] = V[j];
    cudaError_t e = launch_multidot(L, k, w, h->ndof, h->kpart, out, s);
    if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "multidot launch: %s", cudaGetErrorString(e));
    return SEM_OK;
}

// w += sign * sum_j coef[j] V_j (coef on the device)
int axpys(sem_t h, double* w, const double* const* V, int k, const double* coef, double sign, cudaStream_t s) {
    VecList L;
    for (int j = 0; j < k; ++j) L.v[j] = V[j];
    cudaError_t e = launch_multiaxpy(w, L, k, coef, sign, h->ndof, s);
    if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "multiaxpy launch: %s", cudaGetErrorString(e));
    return SEM_OK;
}

int host_norm(sem_t h, const double* a, cudaStream_t s, double& out) {
    SEM_TRY(dots(h, &a, 1, a, h->kscal + KMAX, s));
    double v = 0.0;
    SEM_CK(cudaMemcpyAsync(&v, h->kscal + KMAX, sizeof(double), cudaMemcpyDeviceToHost, s));
    SEM_CK(cudaStreamSynchronize(s));
    out = std::sqrt(v);
    return SEM_OK;
}

// out = sb * b + sx * x + so * Op(u) x  with Op = J (OP_JAC) or J^T (OP_JACT); b may be null
int shifted(sem_t h, int op, const double* u, double so, const double* x, double sx, const double* b, double sb,
            double* out, cudaStream_t s) {
    Epi ep;
    std::memset(&ep, 0, sizeof(ep));
    ep.nonfinite = h->flag;
    ep.out[0] = out;
    ep.alpha[0] = so;
    ep.src[0] = x;
    ep.beta[0][0] = sx;
    ep.nsrc = 1;
    if (b) {
        ep.src[1] = b;
        ep.beta[0][1] = sb;
        ep.nsrc = 2;
    }
    ep.nout = 1;
    ++h->cn_st[3];
    return apply(h, op, u, x, ep, s);
}

// Solve (I - c Op(u)) x = b by restarted GMRES(m) from x = 0 to |b - A x| <= rtol |b|;
// its accumulates the Arnoldi steps.
int gmres(sem_t h, int op, const double* u, double c, const double* b, double* x, cudaStream_t s, long long& its) {
    SEM_TRY(krylov_ws(h));
    const int m = h->krylov_m;
    double* w = kvec(h, m + 1);
    SEM_CK(cudaMemsetAsync(x, 0, vec_bytes(h), s));
    double bnorm = 0.0;
    SEM_TRY(host_norm(h, b, s, bnorm));
    if (bnorm == 0.0) return SEM_OK;
    if (!std::isfinite(bnorm)) return fail(SEM_ERR_NONFINITE, "non-finite right-hand side of a linear solve");
    const double tol = h->krylov_rtol * bnorm;
    double beta = bnorm;
    const double* r = b;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), h1(m + 2), h2(m + 2), y(m);
    long long total = 0;
    for (;;) {
        cudaError_t e = launch_scale(kvec(h, 0), r, 1.0 / beta, h->ndof, s);   // v_0 = r / beta
        if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "scale launch: %s", cudaGetErrorString(e));
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        bool done = false;
        while (j < m && total < h->krylov_maxit) {
            SEM_TRY(shifted(h, op, u, -c, kvec(h, j), 1.0, nullptr, 0.0, w, s));   // w = A v_j
            const double* V[KMAX];
            for (int i = 0; i <= j; ++i) V[i] = kvec(h, i);
            SEM_TRY(dots(h, V, j + 1, w, h->kscal, s));
            SEM_TRY(axpys(h, w, V, j + 1, h->kscal, -1.0, s));
            SEM_TRY(dots(h, V, j + 1, w, h->kscal + KMAX, s));
            SEM_TRY(axpys(h, w, V, j + 1, h->kscal + KMAX, -1.0, s));
            const double* ww = w;
            SEM_TRY(dots(h, &ww, 1, w, h->kscal + KMAX + j + 1, s));
            SEM_CK(cudaMemcpyAsync(h1.data(), h->kscal, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
            SEM_CK(cudaMemcpyAsync(h2.data(), h->kscal + KMAX, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, s));
            SEM_CK(cudaStreamSynchronize(s));
            ++total;
            double* col = &H[0];
            for (int i = 0; i <= j; ++i) col[(size_t)i * m + j] = h1[i] + h2[i];
            const double hn = std::sqrt(std::max(h2[j + 1], 0.0));
            for (int i = 0; i < j; ++i) {   // apply the earlier rotations to column j
                const double a0 = col[(size_t)i * m + j], a1 = col[(size_t)(i + 1) * m + j];
                col[(size_t)i * m + j] = cs[i] * a0 + sn[i] * a1;
                col[(size_t)(i + 1) * m + j] = -sn[i] * a0 + cs[i] * a1;
            }
            const double a0 = col[(size_t)j * m + j];
            const double rr = std::hypot(a0, hn);
            if (!(rr > 0.0) || !std::isfinite(rr)) return fail(SEM_ERR_NONFINITE, "GMRES breakdown (column norm %g)", rr);
            cs[j] = a0 / rr;
            sn[j] = hn / rr;
            col[(size_t)j * m + j] = rr;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++j;
            if (std::fabs(g[j]) <= tol || hn == 0.0) {
                done = true;
                break;
            }
            if (j < m) {
                e = launch_scale(kvec(h, j), w, 1.0 / hn, h->ndof, s);
                if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "scale launch: %s", cudaGetErrorString(e));
            }
        }
        // x += V y with R y = g (the rotated Hessenberg matrix is upper triangular)
        for (int i = j - 1; i >= 0; --i) {
            double acc = g[i];
            for (int l = i + 1; l < j; ++l) acc -= H[(size_t)i * m + l] * y[l];
            y[i] = acc / H[(size_t)i * m + i];
        }
        SEM_CK(cudaMemcpyAsync(h->kscal, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, s));
        const double* V[KMAX];
        for (int i = 0; i < j; ++i) V[i] = kvec(h, i);
        SEM_TRY(axpys(h, x, V, j, h->kscal, 1.0, s));
        if (done) break;
        if (total >= h->krylov_maxit)
            return fail(SEM_ERR_NONFINITE, "GMRES did not reach relative residual %.1e in %d steps", h->krylov_rtol,
                        h->krylov_maxit);
        SEM_TRY(shifted(h, op, u, c, x, -1.0, b, 1.0, w, s));   // restart from r = b - x + c Op x = b - A x
        SEM_TRY(host_norm(h, w, s, beta));
        if (!std::isfinite(beta)) return fail(SEM_ERR_NONFINITE, "non-finite GMRES residual");
        if (beta <= tol) break;
        r = w;
    }
    its += total;
    return SEM_OK;
}

// One CN step u -> u_next by Newton's method (explicit Euler predictor).
int cn_step(sem_t h, double dt, const double* u, double* u_next, cudaStream_t s) {
    double* Fn = vec(h, V_K0);
    double* b = vec(h, V_K0 + 1);
    double* delta = vec(h, V_K0 + 2);
    {   // Fn = F(u), u_next = u + dt Fn
        Epi ep;
        std::memset(&ep, 0, sizeof(ep));
        ep.nonfinite = h->flag;
        ep.out[0] = Fn;
        ep.alpha[0] = 1.0;
        ep.out[1] = u_next;
        ep.alpha[1] = dt;
        ep.src[0] = u;
        ep.beta[1][0] = 1.0;
        ep.nsrc = 1;
        ep.nout = 2;
        ++h->cn_st[3];
        ++h->st[0];
        SEM_TRY(stage_rhs(h, u, ep, s));
    }
    for (int it = 0; it < h->newton_maxit; ++it) {
        {   // b = -R(v) = dt/2 F(v) - v + u + dt/2 Fn
            Epi ep;
            std::memset(&ep, 0, sizeof(ep));
            ep.nonfinite = h->flag;
            ep.out[0] = b;
            ep.alpha[0] = 0.5 * dt;
            ep.src[0] = u_next;
            ep.beta[0][0] = -1.0;
            ep.src[1] = u;
            ep.beta[0][1] = 1.0;
            ep.src[2] = Fn;
            ep.beta[0][2] = 0.5 * dt;
            ep.nsrc = 3;
            ep.nout = 1;
            ++h->cn_st[3];
            ++h->st[0];
            SEM_TRY(stage_rhs(h, u_next, ep, s));
        }
        SEM_TRY(gmres(h, OP_JAC, jac_point(h, u_next), 0.5 * dt, b, delta, s, h->cn_st[1]));
        ++h->cn_st[0];
        const double* Vd = delta;
        SEM_TRY(axpys(h, u_next, &Vd, 1, h->kscal + KSCAL_ONE, 1.0, s));
        double dn = 0.0, vn = 0.0;
        SEM_TRY(host_norm(h, delta, s, dn));
        SEM_TRY(host_norm(h, u_next, s, vn));
        if (!std::isfinite(dn) || !std::isfinite(vn)) return fail(SEM_ERR_NONFINITE, "non-finite Newton iterate");
        if (dn <= h->newton_rtol * std::max(vn, 1.0)) return SEM_OK;
    }
    return fail(SEM_ERR_NONFINITE, "Newton did not converge in %d iterations", h->newton_maxit);
}

// Forward sweep storing every state u_0 .. u_N (the adjoint needs both ends of each step).
int cn_forward(sem_t h, double dt, int nsteps, const double* u0, double* uT, cudaStream_t s) {
    if (f32(h)) return fail(SEM_ERR_ARG, "the Crank-Nicolson scheme runs in the FP64 form only");
    if (h->batch) return fail(SEM_ERR_ARG, "the Crank-Nicolson scheme is not available for batches");
    SEM_TRY(alloc_traj(h, (size_t)nsteps + 1));
    h->have_fwd = false;
    for (int k = 0; k < 4; ++k) h->cn_st[k] = 0;
    h->st[0] = h->st[1] = h->st[2] = 0;
    SEM_CK(cudaMemcpyAsync(h->traj, u0, vec_bytes(h), cudaMemcpyDeviceToDevice, s));
    for (int n = 0; n < nsteps; ++n)
        SEM_TRY(cn_step(h, dt, h->traj + (size_t)n * h->ndof, h->traj + (size_t)(n + 1) * h->ndof, s));
    SEM_CK(cudaMemcpyAsync(uT, h->traj + (size_t)nsteps * h->ndof, vec_bytes(h), cudaMemcpyDeviceToDevice, s));
    h->have_fwd = true;
    h->f_scheme = SEM_CN;
    h->f_nsteps = nsteps;
    h->f_dt = dt;
    h->f_mode = SEM_CKPT_STATES;
    h->f_slots = 0;
    h->f_ckpt.clear();
    return SEM_OK;
}

int cn_adjoint(sem_t h, const double* lamT, double* lam0, cudaStream_t s) {
    const double dt = h->f_dt;
    double* mu = vec(h, V_NU);
    h->cn_st[2] = 0;
    h->st[2] = 0;
    if (lam0 != lamT) SEM_CK(cudaMemcpyAsync(lam0, lamT, vec_bytes(h), cudaMemcpyDeviceToDevice, s));
    for (int n = h->f_nsteps - 1; n >= 0; --n) {
        const double* un1 = h->traj + (size_t)(n + 1) * h->ndof;
        const double* un = h->traj + (size_t)n * h->ndof;
        const long long before = h->cn_st[3];
        SEM_TRY(gmres(h, OP_JACT, jac_point(h, un1), 0.5 * dt, lam0, mu, s, h->cn_st[2]));
        Epi ep;   // lam_n = mu + dt/2 J(u_n)^T mu
        std::memset(&ep, 0, sizeof(ep));
        ep.nonfinite = h->flag;
        ep.out[0] = lam0;
        ep.alpha[0] = 0.5 * dt;
        ep.src[0] = mu;
        ep.beta[0][0] = 1.0;
        ep.nsrc = 1;
        ep.nout = 1;
        ++h->cn_st[3];
        SEM_TRY(apply(h, OP_JACT, jac_point(h, un), mu, ep, s));
        h->st[2] += h->cn_st[3] - before;
    }
    return SEM_OK;
}

// ------------------------------------------------------------------ adaptive stepping
// Sec. 5.1: the step is chosen from a weighted estimate of the local truncation
// error.  Pair: Bogacki-Shampine 3(2); error E = dt sum_i (b_i - bhat_i) k_i with
// k4 = F(u_{n+1}), in the weighted RMS norm with atol + rtol max(|u_n|, |u_{n+1}|);
// controller: accept when err <= 1, next trial dt min(fmax, max(0.2, 0.9 err^(-1/3)))
// with fmax = 5 (1 right after a rejection); the last step ends on the horizon.
// The stage epilogues carry the solution and the error estimate as running sums.
// One device-to-host read of the error norm per attempted step decides it.

// Keep the first `keep` trajectory vectors while growing the buffer to hold nvec.
int grow_traj(sem_t h, size_t nvec, size_t keep, cudaStream_t s) {
    if (h->traj && h->traj_vectors >= nvec) return SEM_OK;
    const size_t vb = vec_bytes(h);
    size_t cap = std::max<size_t>(std::max<size_t>(nvec, 2 * h->traj_vectors), 16);
    if (h->ckpt_budget) cap = std::min(cap, h->ckpt_budget / vb);
    if (cap < nvec) return fail(SEM_ERR_OOM, "adaptive sweep: %zu states exceed the budget of %zu bytes", nvec,
                                h->ckpt_budget);
    double* nb = nullptr;
    cudaError_t e = cudaMalloc((void**)&nb, cap * vb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SEM_ERR_OOM : SEM_ERR_CUDA,
                    "adaptive sweep: trajectory of %zu bytes: %s", cap * vb, cudaGetErrorString(e));
    }
    if (h->traj && keep) SEM_CK(cudaMemcpyAsync(nb, h->traj, keep * vb, cudaMemcpyDeviceToDevice, s));
    SEM_CK(cudaStreamSynchronize(s));
    cudaFree(h->traj);
    h->traj = nb;
    h->traj_vectors = cap;
    return SEM_OK;
}

// One attempted step u -> unext with its error estimate in err (FP64 form).
int bs3_attempt(sem_t h, double dt, const double* u, double* unext, double* err, cudaStream_t s) {
    Tableau T;
    tableau_of(SEM_BS3, T);
    double* Y1 = vec(h, V_STAGE0);
    double* Y2 = vec(h, V_STAGE0 + 1);
    double* acc = vec(h, V_K0);
    for (int i = 0; i < 4; ++i) {
        Epi ep;
        std::memset(&ep, 0, sizeof(ep));
        ep.nonfinite = h->flag;
        const double d = dt * ((i < 3 ? T.b[i] : 0.0) - BS3_BHAT[i]);
        const double* at = i == 0 ? u : (i == 1 ? Y1 : (i == 2 ? Y2 : unext));
        if (i < 2) {   // next stage, running solution, running error
            const int su = add_src(ep, u);
            ep.out[0] = i == 0 ? Y1 : Y2;
            ep.alpha[0] = dt * T.A[i + 1][i];
            ep.beta[0][su] = 1.0;
            const int sa = i == 0 ? su : add_src(ep, acc);
            ep.out[1] = acc;
            ep.alpha[1] = dt * T.b[i];
            ep.beta[1][sa] = 1.0;
            ep.out[2] = err;
            ep.alpha[2] = d;
            if (i > 0) ep.beta[2][add_src(ep, err)] = 1.0;
            ep.nout = 3;
        } else if (i == 2) {   // the solution, running error
            const int sa = add_src(ep, acc);
            ep.out[0] = unext;
            ep.alpha[0] = dt * T.b[2];
            ep.beta[0][sa] = 1.0;
            ep.out[1] = err;
            ep.alpha[1] = d;
            ep.beta[1][add_src(ep, err)] = 1.0;
            ep.nout = 2;
        } else {   // k4 = F(u_{n+1}) enters the error only
            ep.out[0] = err;
            ep.alpha[0] = d;
            ep.beta[0][add_src(ep, err)] = 1.0;
            ep.nout = 1;
        }
        SEM_TRY(stage_rhs(h, at, ep, s));
    }
    return SEM_OK;
}

int adaptive_forward(sem_t h, double T, double dt0, const double* u0, double* uT, cudaStream_t s) {
    if (f32(h)) return fail(SEM_ERR_ARG, "adaptive stepping runs in the FP64 form only");
    const size_t vb = vec_bytes(h);
    h->have_fwd = false;
    SEM_TRY(grow_traj(h, 2, 0, s));
    SEM_CK(cudaMemcpyAsync(h->traj, u0, vb, cudaMemcpyDeviceToDevice, s));
    std::vector<double> dts;
    long long rejected = 0, count = 0;
    double t = 0.0, dt = dt0;
    bool after_reject = false;
    double* err = vec(h, V_K0 + 1);
    if (!h->adapt_buf) {   // partial sums of the error norm and its total
        cudaError_t e = cudaMalloc((void**)&h->adapt_buf, sizeof(double) * (multidot_blocks(h->ndof) + 1));
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->adapt_buf = nullptr;
            return fail(SEM_ERR_OOM, "adaptive sweep workspace: %s", cudaGetErrorString(e));
        }
    }
    double* part = h->adapt_buf + 1;
    double* total = h->adapt_buf;
    while (t < T) {
        if (dts.size() >= 10000000) return fail(SEM_ERR_NONFINITE, "adaptive sweep: more than 1e7 steps");
        const bool last = t + dt >= T * (1.0 - 1e-12);
        const double step = last ? T - t : dt;
        const size_t n = dts.size();
        SEM_TRY(grow_traj(h, n + 2, n + 1, s));
        double* un = h->traj + n * h->ndof;
        double* next = h->traj + (n + 1) * h->ndof;
        SEM_TRY(bs3_attempt(h, step, un, next, err, s));
        count += 4;
        cudaError_t e = launch_wrms_sum(err, un, next, h->adapt_atol, h->adapt_rtol, h->ndof, part, total, s);
        if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "error norm launch: %s", cudaGetErrorString(e));
        double sum = 0.0;
        unsigned flag = 0;
        SEM_CK(cudaMemcpyAsync(&sum, total, sizeof(double), cudaMemcpyDeviceToHost, s));
        SEM_CK(cudaMemcpyAsync(&flag, h->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        SEM_CK(cudaStreamSynchronize(s));
        double enorm = std::sqrt(sum / (double)h->ndof);
        if (flag) {   // a non-finite attempt is rejected like a too-large error
            SEM_CK(cudaMemsetAsync(h->flag, 0, sizeof(unsigned), s));
            enorm = std::numeric_limits<double>::infinity();
        }
        const double fmax = after_reject ? 1.0 : 5.0;
        const double fac = enorm > 0.0 ? std::min(fmax, std::max(0.2, 0.9 * std::pow(enorm, -1.0 / 3.0))) : fmax;
        if (enorm <= 1.0) {
            dts.push_back(step);
            t = last ? T : t + step;
            if (!last) dt = step * fac;
            after_reject = false;
        } else {
            ++rejected;
            after_reject = true;
            dt = step * fac;
            if (!(dt > 1e-14 * T)) return fail(SEM_ERR_NONFINITE, "adaptive sweep: step size underflow at t = %g", t);
        }
    }
    const int N = (int)dts.size();
    SEM_CK(cudaMemcpyAsync(uT, h->traj + (size_t)N * h->ndof, vb, cudaMemcpyDeviceToDevice, s));
    h->have_fwd = true;
    h->f_scheme = SEM_BS3;
    h->f_nsteps = N;
    h->f_dt = dts.back();
    h->f_mode = MODE_ADAPTIVE;
    h->f_slots = 0;
    h->f_ckpt.clear();
    h->f_dts = dts;
    h->f_rejected = rejected;
    h->st[0] = count;
    return SEM_OK;
}

// ------------------------------------------------------------------ batches
template <typename T>
int upload(T** dst, const std::vector<T>& src) {
    cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * std::max<size_t>(src.size(), 1));
    if (e == cudaSuccess && !src.empty())
        e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SEM_ERR_OOM : SEM_ERR_CUDA, "batch tables: %s",
                    cudaGetErrorString(e));
    }
    return SEM_OK;
}

// Work items for a block size: each instance's elements in chunks of threads / NP.
int batch_items(sem_t h, int threads) {
    BatchHost* b = h->batch;
    std::vector<WorkItem> items;
    for (int k = 0; k < b->count; ++k) {
        const BatchInst& in = b->inst[k];
        const int epb = threads / in.NP;
        for (int e0 = 0; e0 < in.nelem; e0 += epb) items.push_back({k, e0, std::min(epb, in.nelem - e0), in.NP});
    }
    cudaFree(b->d_items);
    b->d_items = nullptr;
    SEM_TRY(upload(&b->d_items, items));
    b->nitems = (int)items.size();
    b->threads = threads;
    const size_t smem = batch_elem_smem(threads, OP_JAC);
    int per_sm = std::min<int>(2048 / threads, (int)((227u * 1024u) / std::max<size_t>(smem, 1)));
    per_sm = std::max(1, per_sm);
    b->blocks = std::max(1, std::min(b->nitems, 152 * per_sm));
    return SEM_OK;
}

BatchDev batch_dev(sem_t h) {
    BatchHost* b = h->batch;
    BatchDev d;
    d.inst = b->d_inst;
    d.items = b->d_items;
    d.nitems = b->nitems;
    d.rows = b->d_rows;
    d.nrows = (int)b->rows.size();
    d.mats = b->d_mats;
    return d;
}

int batch_tables(sem_t h) {
    BatchHost* b = h->batch;
    if (b->d_inst) return SEM_OK;
    SEM_TRY(upload(&b->d_inst, b->inst));
    SEM_TRY(upload(&b->d_mats, b->mats));
    SEM_TRY(upload(&b->d_rows, b->rows));
    SEM_TRY(upload(&b->d_row_start, b->row_start));
    std::vector<double> zeros(b->count + 1, 0.0), rz(b->rows.size(), 0.0);
    SEM_TRY(upload(&b->d_J, zeros));
    SEM_TRY(upload(&b->d_rowpart, rz));
    return SEM_OK;
}

// Autotuner: time the batched J^T element pass (the most expensive) for each
// candidate block size and keep the fastest.  Synchronises `s`.
int batch_tune(sem_t h, cudaStream_t s) {
    BatchHost* b = h->batch;
    SEM_TRY(batch_tables(h));
    const int cand[4] = {64, 128, 192, 256};
    cudaEvent_t e0, e1;
    SEM_CK(cudaEventCreate(&e0));
    SEM_CK(cudaEventCreate(&e1));
    SEM_CK(cudaMemsetAsync(vec(h, V_CUR0), 0, 2 * vec_bytes(h), s));
    int best = 128;
    float best_ms = 1e30f;
    for (int ci = 0; ci < 4; ++ci) {
        SEM_TRY(batch_items(h, cand[ci]));
        const BatchDev d = batch_dev(h);
        const size_t smem = batch_elem_smem(cand[ci], OP_JACT);
        float tot = 0.f;
        for (int rep = 0; rep < 4; ++rep) {
            SEM_CK(cudaEventRecord(e0, s));
            cudaError_t e = launch_batch_elem(d, OP_JACT, vec(h, V_CUR0), vec(h, V_CUR1), (double*)h->lvec,
                                              cand[ci], b->blocks, smem, s);
            if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "batched element kernel: %s", cudaGetErrorString(e));
            SEM_CK(cudaEventRecord(e1, s));
            SEM_CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            SEM_CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) tot += ms;
        }
        b->tune_ms[ci] = tot / 3;
        if (tot < best_ms) {
            best_ms = tot;
            best = cand[ci];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return batch_items(h, best);
}

int batch_apply(sem_t h, int op, const double* u, const double* w, const Epi& ep, cudaStream_t s) {
    BatchHost* b = h->batch;
    SEM_TRY(batch_tables(h));
    if (!b->threads) SEM_TRY(batch_tune(h, s));
    const BatchDev d = batch_dev(h);
    long long slot;
    SEM_TRY(prof_begin(h, op, s, slot));
    cudaError_t e = launch_batch_elem(d, op, u, w, (double*)h->lvec, b->threads, b->blocks,
                                      batch_elem_smem(b->threads, op), s);
    if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "batched element kernel: %s", cudaGetErrorString(e));
    SEM_TRY(prof_end(h, slot, s));
    SEM_TRY(prof_begin(h, 3, s, slot, asm_bytes(h, ep)));
    e = launch_batch_assemble(d, (const double*)h->lvec, op != OP_JACT, ep, s);
    if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "batched assembly: %s", cudaGetErrorString(e));
    SEM_TRY(prof_end(h, slot, s));
    return SEM_OK;
}

int batch_objective(sem_t h, const double* u, const double* uo, double* lam, cudaStream_t s) {
    BatchHost* b = h->batch;
    SEM_TRY(batch_tables(h));
    cudaError_t e = launch_batch_objective(batch_dev(h), u, uo, lam, b->d_rowpart, b->d_row_start, b->count,
                                           b->d_J, h->scal, s);
    if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "batched misfit: %s", cudaGetErrorString(e));
    return SEM_OK;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

int sem_create_ex(const sem_opts* o, sem_t* out) {
    if (!out) return fail(SEM_ERR_ARG, "out is null");
    *out = nullptr;
    SEM_TRY(validate(o));
    sem_ctx* h = new sem_ctx();
    h->dim = o->dim;
    h->E = o->E;
    h->N = o->N;
    h->np = o->N + 1;
    h->G = o->E * o->N;
    h->nu = o->nu;
    h->L = o->L > 0 ? o->L : (o->dim == 1 ? 2.0 * M_PI : 1.0);
    h->h = h->L / o->E;
    h->precision = o->precision;
    h->ckpt_mode = o->ckpt_mode;
    h->ckpt_slots = o->ckpt_slots;
    h->ckpt_budget = o->ckpt_budget_bytes;
    semh::gll(h->N, h->xi, h->w);
    semh::derivative(h->xi, h->Dh);
    semh::kernel_matrices(h->w, h->Dh, h->h, h->nu, h->mats);
    h->mw.assign(h->N, 0.0);
    for (int i = 0; i < h->N; ++i) h->mw[i] = h->w[i];
    h->mw[0] = h->w[0] + h->w[h->N];
    h->ndof = h->dim;
    h->nelem = 1;
    h->lvec_elems = h->dim;
    for (int d = 0; d < h->dim; ++d) {
        h->ndof *= (size_t)h->G;
        h->nelem *= h->E;
        h->lvec_elems *= (size_t)h->E * h->np;
    }
    *out = h;
    g_err.clear();
    return SEM_OK;
}

int sem_create(int dim, int E, int N, double nu, sem_t* out) {
    sem_opts o;
    std::memset(&o, 0, sizeof(o));
    o.dim = dim;
    o.E = E;
    o.N = N;
    o.nu = nu;
    return sem_create_ex(&o, out);
}

void sem_destroy(sem_t h) {
    if (!h) return;
    if (h->lvec || h->traj) cudaDeviceSynchronize();
    for (size_t i = 0; i < h->ev_start.size(); ++i) {
        cudaEventDestroy(h->ev_start[i]);
        cudaEventDestroy(h->ev_stop[i]);
    }
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph_stream) cudaStreamDestroy(h->graph_stream);
    prof_graph_release(h);
    cudaFree(h->lvec);
    cudaFree(h->partials);
    cudaFree(h->scal);
    cudaFree(h->flag);
    cudaFree(h->vecs);
    cudaFree(h->traj);
    cudaFree(h->kbasis);
    cudaFree(h->kpart);
    cudaFree(h->kscal);
    cudaFree(h->frozen);
    cudaFree(h->adapt_buf);
    if (h->host_traj) cudaFreeHost(h->host_traj);
    for (int k = 0; k < 3; ++k) {
        if (h->ev_comp[k]) cudaEventDestroy(h->ev_comp[k]);
        if (h->ev_copy[k]) cudaEventDestroy(h->ev_copy[k]);
        if (h->ev_load[k]) cudaEventDestroy(h->ev_load[k]);
        if (h->ev_done[k]) cudaEventDestroy(h->ev_done[k]);
    }
    if (h->cstream) cudaStreamDestroy(h->cstream);
    if (h->batch) {
        BatchHost* b = h->batch;
        cudaFree(b->d_inst);
        cudaFree(b->d_mats);
        cudaFree(b->d_rows);
        cudaFree(b->d_row_start);
        cudaFree(b->d_items);
        cudaFree(b->d_J);
        cudaFree(b->d_rowpart);
        delete b;
    }
    delete h;
}

size_t sem_ndof(sem_t h) { return h ? h->ndof : 0; }

int sem_coords(sem_t h, double* x) {
    if (!h || !x) return fail(SEM_ERR_ARG, "null handle or output");
    if (h->batch) return fail(SEM_ERR_ARG, "sem_coords: use sem_batch_coords for a batch handle");
    for (int g = 0; g < h->G; ++g) {
        const int e = g / h->N, i = g % h->N;
        x[g] = e * h->h + (h->xi[i] + 1.0) * h->h / 2.0;
    }
    return SEM_OK;
}

// FP32 form, standalone apply: the caller's doubles become float pairs once
// (integer split, one pass over the unknowns) so that the element kernel reads
// pair planes; the result is widened back to doubles by the assembly.  J^T reads
// only the hi plane of v (Z = v / k in FP32), so only that plane is written.
static int standalone(sem_t h, int op, const double* u, const double* w, double* out, cudaStream_t s) {
    if (!f32(h)) return apply(h, op, u, w, epi_plain(out, nullptr), s);
    cudaError_t e = launch_f64_to_f2(u, fl(vec(h, V_CUR0)), h->ndof, s);
    if (e == cudaSuccess && w) e = launch_f64_to_f2(w, fl(vec(h, V_CUR1)), h->ndof, s, op == OP_JACT);
    if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "conversion launch: %s", cudaGetErrorString(e));
    return apply(h, op, vec(h, V_CUR0), w ? vec(h, V_CUR1) : nullptr, epi_plain(out, nullptr), s, true);
}

int sem_rhs(sem_t h, const double* u, double* f, void* stream) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    SEM_TRY(check_state_ptr(u, "u"));
    SEM_TRY(check_state_ptr(f, "f"));
    if (overlap(u, f, vec_bytes(h))) return fail(SEM_ERR_ALIAS, "f overlaps u");
    SEM_TRY(ensure_workspace(h));
    return standalone(h, OP_RHS, u, nullptr, f, (cudaStream_t)stream);
}

int sem_jac_apply(sem_t h, const double* u, const double* w, double* jw, void* stream) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    SEM_TRY(check_state_ptr(u, "u"));
    SEM_TRY(check_state_ptr(w, "w"));
    SEM_TRY(check_state_ptr(jw, "jw"));
    if (overlap(u, jw, vec_bytes(h)) || overlap(w, jw, vec_bytes(h))) return fail(SEM_ERR_ALIAS, "jw overlaps an input");
    SEM_TRY(ensure_workspace(h));
    return standalone(h, OP_JAC, u, w, jw, (cudaStream_t)stream);
}

int sem_jacT_apply(sem_t h, const double* u, const double* v, double* jtv, void* stream) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    SEM_TRY(check_state_ptr(u, "u"));
    SEM_TRY(check_state_ptr(v, "v"));
    SEM_TRY(check_state_ptr(jtv, "jtv"));
    if (overlap(u, jtv, vec_bytes(h)) || overlap(v, jtv, vec_bytes(h))) return fail(SEM_ERR_ALIAS, "jtv overlaps an input");
    SEM_TRY(ensure_workspace(h));
    return standalone(h, OP_JACT, u, v, jtv, (cudaStream_t)stream);
}

int sem_rk_forward(sem_t h, int scheme, double dt, int nsteps, const double* u0, double* uT, void* stream) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    cudaStream_t s = (cudaStream_t)stream;
    SEM_TRY(ensure_workspace(h));
    SEM_CK(cudaMemsetAsync(h->flag, 0, sizeof(unsigned), s));
    SEM_TRY(forward_impl(h, scheme, dt, nsteps, u0, uT, s));
    return check_flag(h, s, "forward");
}

int sem_rk_adjoint(sem_t h, const double* lamT, double* lam0, void* stream) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    cudaStream_t s = (cudaStream_t)stream;
    if (h->flag) SEM_CK(cudaMemsetAsync(h->flag, 0, sizeof(unsigned), s));
    SEM_TRY(adjoint_impl(h, lamT, lam0, s));
    return check_flag(h, s, "adjoint");
}

int sem_objective(sem_t h, const double* u, const double* uo, double* J_host, double* lam, void* stream) {
    if (!h || !J_host) return fail(SEM_ERR_ARG, "null handle or J_host");
    SEM_TRY(check_state_ptr(u, "u"));
    SEM_TRY(check_state_ptr(uo, "u_obs"));
    if (lam) {
        SEM_TRY(check_state_ptr(lam, "lam"));
        if (overlap(lam, u, vec_bytes(h)) || overlap(lam, uo, vec_bytes(h))) return fail(SEM_ERR_ALIAS, "lam overlaps an input");
    }
    SEM_TRY(ensure_workspace(h));
    cudaStream_t s = (cudaStream_t)stream;
    SEM_TRY(objective_impl(h, u, uo, lam, s));
    SEM_CK(cudaMemcpyAsync(J_host, h->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    SEM_CK(cudaStreamSynchronize(s));
    return SEM_OK;
}

// The launch sequence of one gradient evaluation (no host synchronisation inside).
static int objective_grad_launches(sem_t h, int scheme, double dt, int nsteps, const double* u0, const double* uo,
                                   double* grad, cudaStream_t s) {
    double* uN = vec(h, V_UN);
    SEM_CK(cudaMemsetAsync(h->flag, 0, sizeof(unsigned), s));
    SEM_TRY(forward_impl(h, scheme, dt, nsteps, u0, uN, s, true));
    if (f32(h)) {
        SEM_TRY(objective_impl(h, uN, uo, vec(h, V_LAM), s, true));
        SEM_TRY(adjoint_impl(h, nullptr, grad, s, true));
    } else {
        SEM_TRY(objective_impl(h, uN, uo, grad, s));
        SEM_TRY(adjoint_impl(h, grad, grad, s));
    }
    return SEM_OK;
}

// Record the gradient evaluation into a CUDA graph on a private stream (after
// every allocation it needs), then replay it on `s` while the arguments match.
static int objective_grad_graph(sem_t h, int scheme, double dt, int nsteps, const double* u0, const double* uo,
                                double* grad, cudaStream_t s) {
    sem_ctx::GraphKey key{scheme, nsteps, dt, u0, uo, grad};
    if (!h->graph_exec || !(h->graph_key == key)) {
        Tableau T;
        if (!tableau_of(scheme, T)) return fail(SEM_ERR_ARG, "unknown RK scheme %d", scheme);
        int mode, slots;
        SEM_TRY(choose_mode(h, T.s, nsteps, mode, slots));
        if (mode == SEM_CKPT_BINOMIAL && slots > nsteps) slots = nsteps;
        if (!h->frozen)
            SEM_TRY(alloc_traj(h, mode == SEM_CKPT_STAGES ? (size_t)nsteps * T.s
                                     : (mode == SEM_CKPT_STATES ? (size_t)nsteps : (size_t)slots)));
        if (h->batch && !h->batch->threads) SEM_TRY(batch_tune(h, s));
        if (!h->graph_stream) SEM_CK(cudaStreamCreateWithFlags(&h->graph_stream, cudaStreamNonBlocking));
        SEM_CK(cudaStreamSynchronize(s));
        h->fixed_mode = mode;
        h->fixed_slots = slots;
        if (h->graph_exec) {
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
        }
        prof_graph_release(h);
        for (int i = 0; i < 4; ++i) h->prof_tick[i] = 0;
        cudaGraph_t g = nullptr;
        SEM_CK(cudaStreamBeginCapture(h->graph_stream, cudaStreamCaptureModeThreadLocal));
        h->capturing = true;
        const int rc = objective_grad_launches(h, scheme, dt, nsteps, u0, uo, grad, h->graph_stream);
        h->capturing = false;
        cudaError_t ec = cudaStreamEndCapture(h->graph_stream, &g);
        h->fixed_mode = -1;
        if (rc != SEM_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ec != cudaSuccess) return fail(SEM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec));
        if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
        ec = cudaGraphInstantiate(&h->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (ec != cudaSuccess) return fail(SEM_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(ec));
        h->graph_key = key;
    }
    SEM_CK(cudaGraphLaunch(h->graph_exec, s));
    ++h->graph_replays;
    return SEM_OK;
}

int sem_objective_grad(sem_t h, int scheme, double dt, int nsteps, const double* u0, const double* uo,
                       double* J_host, double* grad, void* stream) {
    if (!h || !J_host) return fail(SEM_ERR_ARG, "null handle or J_host");
    SEM_TRY(check_state_ptr(u0, "u0"));
    SEM_TRY(check_state_ptr(uo, "u_obs"));
    SEM_TRY(check_state_ptr(grad, "grad"));
    if (overlap(grad, u0, vec_bytes(h)) || overlap(grad, uo, vec_bytes(h)))
        return fail(SEM_ERR_ALIAS, "grad overlaps an input");
    if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 1) return fail(SEM_ERR_ARG, "dt > 0 and nsteps >= 1");
    SEM_TRY(ensure_workspace(h));
    cudaStream_t s = (cudaStream_t)stream;
    // the implicit scheme synchronises with the host inside its solves, and the two-level
    // store runs a second stream: neither is captured
    bool graph = h->graph_on && scheme != SEM_CN && !adaptive(h, scheme);
    if (graph) {
        Tableau T;
        int mode, slots;
        if (!tableau_of(scheme, T)) return fail(SEM_ERR_ARG, "unknown time scheme %d", scheme);
        SEM_TRY(choose_mode(h, T.s, nsteps, mode, slots));
        if (mode == SEM_CKPT_TWO_LEVEL && !h->frozen) graph = false;
    }
    if (graph) SEM_TRY(objective_grad_graph(h, scheme, dt, nsteps, u0, uo, grad, s));
    else SEM_TRY(objective_grad_launches(h, scheme, dt, nsteps, u0, uo, grad, s));
    unsigned f = 0;
    SEM_CK(cudaMemcpyAsync(J_host, h->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    SEM_CK(cudaMemcpyAsync(&f, h->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SEM_CK(cudaStreamSynchronize(s));
    if (graph && h->prof) SEM_TRY(prof_graph_accumulate(h));
    if (f || !std::isfinite(*J_host)) return fail(SEM_ERR_NONFINITE, "non-finite values in the gradient evaluation");
    return SEM_OK;
}

int sem_set_graph(sem_t h, int enable) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    h->graph_on = enable != 0;
    if (!h->graph_on && h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
        h->graph_key = sem_ctx::GraphKey{-1, 0, 0.0, nullptr, nullptr, nullptr};
        prof_graph_release(h);
    }
    return SEM_OK;
}

long long sem_graph_replays(sem_t h) { return h ? h->graph_replays : -1; }

int sem_ckpt_plan(int nsteps, int slots, long long* advances) {
    if (nsteps < 1 || slots < 0 || !advances) return fail(SEM_ERR_ARG, "nsteps >= 1, slots >= 0, advances != null");
    semh::CkptPlanner P(nsteps, slots);
    *advances = P.cost(nsteps, slots);
    return SEM_OK;
}

int sem_sweep_stats(sem_t h, long long* out3) {
    if (!h || !out3) return fail(SEM_ERR_ARG, "null handle or output");
    for (int i = 0; i < 3; ++i) out3[i] = h->st[i];
    return SEM_OK;
}

int sem_set_advection(sem_t h, const double* a, void* stream) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    cudaStream_t s = (cudaStream_t)stream;
    // a recorded gradient graph and a recorded forward sweep belong to the previous equation
    if (h->graph_exec) {
        SEM_CK(cudaStreamSynchronize(s));
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
        h->graph_key = sem_ctx::GraphKey{-1, 0, 0.0, nullptr, nullptr, nullptr};
        prof_graph_release(h);
    }
    h->have_fwd = false;
    if (!a) {
        if (h->frozen) {
            SEM_CK(cudaStreamSynchronize(s));
            cudaFree(h->frozen);
            h->frozen = nullptr;
        }
        return SEM_OK;
    }
    SEM_TRY(check_state_ptr(a, "a"));
    SEM_TRY(ensure_workspace(h));
    if (!h->frozen) {
        cudaError_t e = cudaMalloc((void**)&h->frozen, vec_bytes(h));
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->frozen = nullptr;
            return fail(e == cudaErrorMemoryAllocation ? SEM_ERR_OOM : SEM_ERR_CUDA, "advecting field: %s",
                        cudaGetErrorString(e));
        }
    }
    if (f32(h)) {
        cudaError_t e = launch_f64_to_f2(a, fl(h->frozen), h->ndof, s);
        if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "conversion launch: %s", cudaGetErrorString(e));
    } else {
        SEM_CK(cudaMemcpyAsync(h->frozen, a, vec_bytes(h), cudaMemcpyDeviceToDevice, s));
    }
    return SEM_OK;
}

int sem_set_contraction(sem_t h, int mode) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    if (mode != SEM_CONTRACT_CUDA_CORE && mode != SEM_CONTRACT_TENSOR)
        return fail(SEM_ERR_ARG, "unknown contraction mode %d", mode);
    if (mode == SEM_CONTRACT_TENSOR &&
        (h->batch || h->dim != 3 || h->np != 16 || h->precision == SEM_PREC_FP64_DF))
        return fail(SEM_ERR_ARG, "tensor-core contractions need a 3D handle of order 15 in the FP64 or FP32-bulk form");
    if (h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
    }
    h->contraction = mode;
    return SEM_OK;
}

int sem_set_dependent_launch(int enable) {
    semk::set_pdl(enable != 0);
    return SEM_OK;
}

int sem_launch_count(sem_t h, long long* launches) {
    if (!h || !launches) return fail(SEM_ERR_ARG, "null handle or output");
    *launches = h->nlaunch;
    return SEM_OK;
}

int sem_set_adaptive(sem_t h, double atol, double rtol) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    if (!(atol >= 0.0) || !(rtol >= 0.0) || !std::isfinite(atol) || !std::isfinite(rtol))
        return fail(SEM_ERR_ARG, "tolerances must be finite and >= 0");
    if (f32(h) && (atol > 0.0 || rtol > 0.0)) return fail(SEM_ERR_ARG, "adaptive stepping runs in the FP64 form only");
    h->adapt_atol = atol;
    h->adapt_rtol = rtol;
    return SEM_OK;
}

int sem_adaptive_steps(sem_t h, int* accepted, int* rejected, double* dts, int cap) {
    if (!h || !accepted || !rejected || cap < 0 || (cap > 0 && !dts)) return fail(SEM_ERR_ARG, "bad arguments");
    const bool ok = h->have_fwd && h->f_mode == MODE_ADAPTIVE;
    *accepted = ok ? (int)h->f_dts.size() : 0;
    *rejected = ok ? (int)h->f_rejected : 0;
    for (int i = 0; ok && i < cap && i < *accepted; ++i) dts[i] = h->f_dts[i];
    return SEM_OK;
}

int sem_set_host_tier(sem_t h, size_t host_bytes) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    if (h->host_traj && host_bytes < h->host_vectors * vec_bytes(h)) {
        if (h->cstream) SEM_CK(cudaStreamSynchronize(h->cstream));
        SEM_CK(cudaDeviceSynchronize());
        cudaFreeHost(h->host_traj);
        h->host_traj = nullptr;
        h->host_vectors = 0;
        if (h->f_mode == SEM_CKPT_TWO_LEVEL) h->have_fwd = false;
    }
    h->host_budget = host_bytes;
    return SEM_OK;
}

int sem_trajectory_info(sem_t h, long long* out4) {
    if (!h || !out4) return fail(SEM_ERR_ARG, "null handle or output");
    out4[0] = out4[1] = out4[2] = out4[3] = 0;
    if (!h->have_fwd || h->f_mode == MODE_LINEAR) return SEM_OK;
    if (h->f_mode == MODE_ADAPTIVE) {
        out4[0] = SEM_CKPT_STATES;
        out4[1] = h->f_nsteps + 1;
        return SEM_OK;
    }
    Tableau T;
    const int stages = h->f_scheme == SEM_CN ? 1 : (tableau_of(h->f_scheme, T) ? T.s : 1);
    out4[0] = h->f_mode;
    if (h->f_scheme == SEM_CN) out4[1] = h->f_nsteps + 1;
    else if (h->f_mode == SEM_CKPT_STAGES) out4[1] = (long long)h->f_nsteps * stages;
    else if (h->f_mode == SEM_CKPT_STATES) out4[1] = h->f_nsteps;
    else if (h->f_mode == SEM_CKPT_TWO_LEVEL) {
        out4[1] = h->f_ndev;
        out4[2] = h->f_nsteps - h->f_ndev;
    } else out4[3] = h->f_slots;
    return SEM_OK;
}

int sem_set_solver(sem_t h, double newton_rtol, double krylov_rtol, int krylov_m, int krylov_maxit) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    if (!(newton_rtol > 0.0) || !(krylov_rtol > 0.0) || krylov_m < 1 || krylov_m > KMAX - 2 || krylov_maxit < 1)
        return fail(SEM_ERR_ARG, "tolerances must be > 0, 1 <= krylov_m <= %d, krylov_maxit >= 1", KMAX - 2);
    if (krylov_m != h->krylov_m) {
        if (h->kbasis) SEM_CK(cudaDeviceSynchronize());
        cudaFree(h->kbasis);
        cudaFree(h->kpart);
        cudaFree(h->kscal);
        h->kbasis = nullptr;
        h->kpart = h->kscal = nullptr;
    }
    h->newton_rtol = newton_rtol;
    h->krylov_rtol = krylov_rtol;
    h->krylov_m = krylov_m;
    h->krylov_maxit = krylov_maxit;
    return SEM_OK;
}

int sem_solver_stats(sem_t h, long long* out4) {
    if (!h || !out4) return fail(SEM_ERR_ARG, "null handle or output");
    for (int i = 0; i < 4; ++i) out4[i] = h->cn_st[i];
    return SEM_OK;
}

int sem_profile(sem_t h, int every) {
    if (!h || every < 0) return fail(SEM_ERR_ARG, "null handle or negative sampling period");
    if (!every) SEM_TRY(prof_drain(h));
    h->prof = every;
    for (int i = 0; i < 4; ++i) h->prof_tick[i] = 0;
    return SEM_OK;
}

int sem_profile_read(sem_t h, double* ms4, long long* count4, double* bytes4, int reset) {
    if (!h || !ms4 || !count4) return fail(SEM_ERR_ARG, "null handle or output");
    SEM_TRY(prof_drain(h));
    for (int i = 0; i < 4; ++i) {
        ms4[i] = h->prof_ms[i];
        count4[i] = h->prof_n[i];
        if (bytes4) bytes4[i] = h->prof_bytes[i];
        if (reset) {
            h->prof_ms[i] = 0;
            h->prof_n[i] = 0;
            h->prof_bytes[i] = 0;
        }
    }
    return SEM_OK;
}

int sem_batch_create(int count, const int* E, const int* N, const double* nu, const sem_opts* common,
                     sem_t* out) {
    if (!out) return fail(SEM_ERR_ARG, "out is null");
    *out = nullptr;
    if (count < 1 || !E || !N || !nu) return fail(SEM_ERR_ARG, "count >= 1 and non-null E, N, nu");
    const int precision = common ? common->precision : SEM_PREC_FP64;
    if (precision != SEM_PREC_FP64) return fail(SEM_ERR_ARG, "batches support the FP64 form");
    const double Lbox = (common && common->L > 0) ? common->L : 1.0;
    BatchHost* b = new BatchHost();
    b->count = count;
    size_t off = 0, loff = 0, nel = 0;
    for (int k = 0; k < count; ++k) {
        const int np = N[k] + 1;
        if (E[k] < 1 || !batch_np_supported(np) || !(nu[k] >= 0.0) || !std::isfinite(nu[k]) ||
            (long long)E[k] * N[k] > 65535) {
            delete b;
            return fail(SEM_ERR_ARG, "instance %d: need E >= 1, N in {3, 5, 7, 9}, finite nu >= 0 (got E=%d N=%d)", k,
                        E[k], N[k]);
        }
        BatchInst in;
        std::memset(&in, 0, sizeof(in));
        in.E = E[k];
        in.N = N[k];
        in.NP = np;
        in.G = E[k] * N[k];
        in.nelem = E[k] * E[k];
        in.GD = (unsigned)in.G * in.G;
        in.off = (unsigned)off;
        in.loff = loff;
        const double hk = Lbox / E[k];
        std::vector<double> xi, w, Dh, mats;
        semh::gll(N[k], xi, w);
        semh::derivative(xi, Dh);
        semh::kernel_matrices(w, Dh, hk, nu[k], mats);
        for (int i = 0; i < N[k]; ++i) in.mw[i] = w[i];
        in.mw[0] = w[0] + w[N[k]];
        in.scale = (hk / 2.0) * (hk / 2.0);
        for (in.divN_shift = 16; in.divN_shift <= 31; ++in.divN_shift) {
            in.divN_mul = (unsigned)(((1ull << in.divN_shift) + N[k] - 1) / N[k]);
            bool ok = true;
            for (unsigned g = 0; g < (unsigned)in.G && ok; ++g)
                ok = (unsigned)(((unsigned long long)g * in.divN_mul) >> in.divN_shift) == g / (unsigned)N[k];
            if (ok) break;
        }
        const size_t moff = (b->mats.size() + 15) & ~(size_t)15;
        const size_t msize = np == 4 ? sizeof(OpMats<double, 4>) : np == 6 ? sizeof(OpMats<double, 6>)
                           : np == 8 ? sizeof(OpMats<double, 8>) : sizeof(OpMats<double, 10>);
        b->mats.resize(moff + msize);
        if (np == 4) fill_opmats<4>(b->mats.data() + moff, mats.data());
        else if (np == 6) fill_opmats<6>(b->mats.data() + moff, mats.data());
        else if (np == 8) fill_opmats<8>(b->mats.data() + moff, mats.data());
        else fill_opmats<10>(b->mats.data() + moff, mats.data());
        in.mats_off = (unsigned)moff;
        b->inst.push_back(in);
        b->row_start.push_back((int)b->rows.size());
        for (int c = 0; c < 2; ++c)
            for (int gy = 0; gy < in.G; ++gy) b->rows.push_back({k, c, gy});
        off += 2 * (size_t)in.G * in.G;
        loff += (size_t)in.nelem * 2 * np * np;
        nel += in.nelem;
        if (off > 2147483647u) {
            delete b;
            return fail(SEM_ERR_ARG, "batch too large: more than 2^31-1 unknowns");
        }
    }
    b->row_start.push_back((int)b->rows.size());
    b->J.assign(count, 0.0);
    sem_ctx* h = new sem_ctx();
    h->batch = b;
    h->dim = 2;
    h->precision = SEM_PREC_FP64;
    h->ckpt_mode = common ? common->ckpt_mode : SEM_CKPT_AUTO;
    h->ckpt_slots = common ? common->ckpt_slots : 0;
    h->ckpt_budget = common ? common->ckpt_budget_bytes : 0;
    h->ndof = off;
    h->lvec_elems = loff;
    h->nelem = (int)nel;
    h->E = b->inst[0].E;
    h->N = b->inst[0].N;
    h->np = b->inst[0].NP;
    h->G = b->inst[0].G;
    h->L = Lbox;
    h->h = Lbox / h->E;
    *out = h;
    g_err.clear();
    return SEM_OK;
}

int sem_batch_count(sem_t h) { return (h && h->batch) ? h->batch->count : 0; }

int sem_batch_layout(sem_t h, int k, size_t* offset, size_t* ndof) {
    if (!h || !h->batch || k < 0 || k >= h->batch->count || !offset || !ndof)
        return fail(SEM_ERR_ARG, "batch handle, 0 <= k < count and non-null outputs");
    const BatchInst& in = h->batch->inst[k];
    *offset = in.off;
    *ndof = 2 * (size_t)in.G * in.G;
    return SEM_OK;
}

int sem_batch_coords(sem_t h, int k, double* x) {
    if (!h || !h->batch || k < 0 || k >= h->batch->count || !x)
        return fail(SEM_ERR_ARG, "batch handle, 0 <= k < count and a non-null output");
    const BatchInst& in = h->batch->inst[k];
    std::vector<double> xi, w;
    semh::gll(in.N, xi, w);
    const double hk = h->L / in.E;
    for (int g = 0; g < in.G; ++g) x[g] = (g / in.N) * hk + (xi[g % in.N] + 1.0) * hk / 2.0;
    return SEM_OK;
}

int sem_batch_autotune(sem_t h, double* ms4, int* threads, void* stream) {
    if (!h || !h->batch) return fail(SEM_ERR_ARG, "batch handle required");
    SEM_TRY(ensure_workspace(h));
    SEM_TRY(batch_tune(h, (cudaStream_t)stream));
    if (ms4)
        for (int i = 0; i < 4; ++i) ms4[i] = h->batch->tune_ms[i];
    if (threads) *threads = h->batch->threads;
    return SEM_OK;
}

int sem_batch_objective_grad(sem_t h, int scheme, double dt, int nsteps, const double* u0, const double* uo,
                             double* J_host, double* grad, void* stream) {
    if (!h || !h->batch || !J_host) return fail(SEM_ERR_ARG, "batch handle and J_host required");
    double Jtot = 0.0;
    SEM_TRY(sem_objective_grad(h, scheme, dt, nsteps, u0, uo, &Jtot, grad, stream));
    SEM_CK(cudaMemcpy(J_host, h->batch->d_J, sizeof(double) * h->batch->count, cudaMemcpyDeviceToHost));
    return SEM_OK;
}

const char* sem_last_error(void) { return g_err.c_str(); }

}  // extern "C"

int semk::max_np(int D, bool fp32) { return (void)D, (void)fp32, 16; }

// Read-only view of a handle for entry points defined in other translation units.
int semk::handle_view(sem_t h, HandleView* v) {
    if (!h || !v) return SEM_ERR_ARG;
    v->dim = h->dim;
    v->E = h->E;
    v->N = h->N;
    v->G = h->G;
    v->np = h->np;
    v->nelem = h->nelem;
    v->ndof = h->ndof;
    v->lvec_elems = h->lvec_elems;
    v->fp32 = h->precision == SEM_PREC_FP32_BULK;
    v->dfloat = h->precision == SEM_PREC_FP64_DF;
    v->batch = h->batch != nullptr;
    v->mats = v->batch ? nullptr : h->mats.data();
    return SEM_OK;
}

void semk::set_error(const char* msg) { g_err = msg; }
