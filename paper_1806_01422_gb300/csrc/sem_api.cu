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
#include <string>
#include <vector>

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
        if (e_ != cudaSuccess) return fail(SEM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
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
    return false;
}

}  // namespace

struct sem_ctx {
    int dim = 0, E = 0, N = 0, np = 0, G = 0;
    int precision = SEM_PREC_FP64, ckpt_mode = SEM_CKPT_AUTO, ckpt_slots = 0;
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
    double* traj = nullptr;
    size_t traj_vectors = 0;
    // last forward sweep
    bool have_fwd = false;
    int f_scheme = 0, f_nsteps = 0, f_mode = 0, f_slots = 0;
    double f_dt = 0;
    std::vector<int> f_ckpt;
    long long st[3] = {0, 0, 0};  // forward F applies, adjoint F applies, adjoint J^T applies
    // opt-in kernel timing: event pairs per launch, drained when the pool fills
    int prof = 0;                 // 0: off; n: time one apply in n per kind
    long long prof_tick[4] = {0, 0, 0, 0};
    std::vector<cudaEvent_t> ev_start, ev_stop;
    std::vector<int> ev_kind;
    size_t ev_used = 0;
    double prof_ms[4] = {0, 0, 0, 0};
    long long prof_n[4] = {0, 0, 0, 0};
};

namespace {

// work vector roles inside sem_ctx::vecs
enum { V_K0 = 0, V_STAGE0 = 4, V_CUR0 = 7, V_CUR1 = 8, V_NU = 9, V_UN = 10, NVEC = 11 };

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
    if (o->precision != SEM_PREC_FP64 && o->precision != SEM_PREC_FP32_BULK)
        return fail(SEM_ERR_ARG, "unknown precision %d", o->precision);
    if (o->ckpt_mode < SEM_CKPT_AUTO || o->ckpt_mode > SEM_CKPT_BINOMIAL)
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
    }
    h->ev_used = 0;
    return SEM_OK;
}

// Returns the index of the event pair to record around one launch (-1: profiling off).
int prof_begin(sem_t h, int kind, cudaStream_t s, long long& slot) {
    slot = -1;
    if (!h->prof) return SEM_OK;
    if (h->prof_tick[kind]++ % h->prof != 0) return SEM_OK;
    if (h->ev_start.empty()) {
        h->ev_start.resize(PROF_POOL);
        h->ev_stop.resize(PROF_POOL);
        h->ev_kind.resize(PROF_POOL);
        for (size_t i = 0; i < PROF_POOL; ++i) {
            SEM_CK(cudaEventCreate(&h->ev_start[i]));
            SEM_CK(cudaEventCreate(&h->ev_stop[i]));
        }
    }
    if (h->ev_used == PROF_POOL) SEM_TRY(prof_drain(h));
    slot = (long long)h->ev_used++;
    h->ev_kind[slot] = kind;
    SEM_CK(cudaEventRecord(h->ev_start[slot], s));
    return SEM_OK;
}

int prof_end(sem_t h, long long slot, cudaStream_t s) {
    if (slot >= 0) SEM_CK(cudaEventRecord(h->ev_stop[slot], s));
    return SEM_OK;
}

// One operator apply: element kernel into the element-local buffer, then the
// gather-scatter sum with the given epilogue.
int apply(sem_t h, int op, const double* u, const double* w, const Epi& ep, cudaStream_t s) {
    ElemArgs a;
    a.u = u;
    a.w = w;
    a.lvec = h->lvec;
    a.E = h->E;
    a.N = h->N;
    a.G = h->G;
    a.nelem = h->nelem;
    const bool f32 = h->precision == SEM_PREC_FP32_BULK;
    long long slot;
    SEM_TRY(prof_begin(h, op, s, slot));
    cudaError_t e;
    if (h->dim == 1) e = f32 ? launch_elem<float, 1>(h->np, op, h->mats.data(), a, s) : launch_elem<double, 1>(h->np, op, h->mats.data(), a, s);
    else if (h->dim == 2) e = f32 ? launch_elem<float, 2>(h->np, op, h->mats.data(), a, s) : launch_elem<double, 2>(h->np, op, h->mats.data(), a, s);
    else e = f32 ? launch_elem<float, 3>(h->np, op, h->mats.data(), a, s) : launch_elem<double, 3>(h->np, op, h->mats.data(), a, s);
    if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "element kernel launch: %s", cudaGetErrorString(e));
    SEM_TRY(prof_end(h, slot, s));
    AsmArgs aa;
    aa.D = h->dim;
    aa.E = h->E;
    aa.N = h->N;
    aa.G = h->G;
    aa.NP = h->np;
    aa.GD = (unsigned)(h->ndof / h->dim);
    aa.ndof = (unsigned)h->ndof;
    aa.scale_mult = op != OP_JACT;
    SEM_TRY(prof_begin(h, 3, s, slot));
    e = launch_assemble(f32, h->lvec, aa, ep, s);
    if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "assembly launch: %s", cudaGetErrorString(e));
    SEM_TRY(prof_end(h, slot, s));
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
int rk_stages(sem_t h, const Tableau& T, double dt, const double* un, double* const* Y, double* unext,
              cudaStream_t s, long long& count) {
    const int last = unext ? T.s - 1 : T.s - 2;
    for (int i = 0; i <= last; ++i) {
        const double* Yi = i == 0 ? un : Y[i];
        Epi ep;
        std::memset(&ep, 0, sizeof(ep));
        ep.nonfinite = h->flag;
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
        SEM_TRY(apply(h, OP_RHS, Yi, nullptr, ep, s));
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
                    cudaStream_t s, long long& count) {
    double* nu = vec(h, V_NU);
    for (int i = T.s - 1; i >= 0; --i) {
        Epi ep;
        std::memset(&ep, 0, sizeof(ep));
        ep.nonfinite = h->flag;
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
            const double c = dt * T.b[T.s - 1];
            ep.out[1] = nu;
            ep.alpha[1] = c;
            for (int m = 0; m < ep.nsrc; ++m) ep.beta[1][m] = c * ep.beta[0][m];
            ep.nout = 2;
        }
        SEM_TRY(apply(h, OP_JACT, Y[i], nu, ep, s));
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

// Storage mode for a sweep of nsteps steps of an s-stage scheme.
int choose_mode(sem_t h, int s, int nsteps, int& mode, int& slots) {
    mode = h->ckpt_mode;
    slots = h->ckpt_slots;
    if (mode != SEM_CKPT_AUTO) return SEM_OK;
    size_t budget = h->ckpt_budget;
    if (!budget) {
        // no explicit budget: the free device memory (plus the trajectory buffer
        // this handle would release) minus 4 GiB of headroom for other users
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            fr = 0;
        }
        fr += h->traj ? h->traj_vectors * vec_bytes(h) : 0;
        const size_t headroom = (size_t)4 << 30;
        budget = fr > headroom ? fr - headroom : fr / 2;
    }
    const size_t v = vec_bytes(h);
    if ((size_t)nsteps * s * v <= budget) mode = SEM_CKPT_STAGES;
    else if ((size_t)nsteps * v <= budget) mode = SEM_CKPT_STATES;
    else {
        mode = SEM_CKPT_BINOMIAL;
        slots = (int)(budget / v);
        if (slots < 1) return fail(SEM_ERR_OOM, "not even one checkpoint slot fits in %zu bytes", budget);
    }
    return SEM_OK;
}

int check_flag(sem_t h, cudaStream_t s, const char* what) {
    unsigned f = 0;
    SEM_CK(cudaMemcpyAsync(&f, h->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SEM_CK(cudaStreamSynchronize(s));
    if (f) return fail(SEM_ERR_NONFINITE, "non-finite values in the %s sweep", what);
    return SEM_OK;
}

int forward_impl(sem_t h, int scheme, double dt, int nsteps, const double* u0, double* uT, cudaStream_t s) {
    Tableau T;
    if (!tableau_of(scheme, T)) return fail(SEM_ERR_ARG, "unknown RK scheme %d", scheme);
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(SEM_ERR_ARG, "dt must be finite and > 0");
    if (nsteps < 1) return fail(SEM_ERR_ARG, "nsteps must be >= 1");
    SEM_TRY(check_state_ptr(u0, "u0"));
    SEM_TRY(check_state_ptr(uT, "uT"));
    if (overlap(u0, uT, vec_bytes(h))) return fail(SEM_ERR_ALIAS, "uT overlaps u0");
    SEM_TRY(ensure_workspace(h));
    int mode, slots;
    SEM_TRY(choose_mode(h, T.s, nsteps, mode, slots));
    if (mode == SEM_CKPT_BINOMIAL && slots > nsteps) slots = nsteps;
    const size_t nvec = mode == SEM_CKPT_STAGES ? (size_t)nsteps * T.s : (mode == SEM_CKPT_STATES ? (size_t)nsteps : (size_t)slots);
    SEM_TRY(alloc_traj(h, nvec));
    h->have_fwd = false;
    const size_t vb = vec_bytes(h);
    double* Yw[4] = {nullptr, vec(h, V_STAGE0), vec(h, V_STAGE0 + 1), vec(h, V_STAGE0 + 2)};
    long long count = 0;
    std::vector<int> ckpt;
    if (mode == SEM_CKPT_STAGES) {
        SEM_CK(cudaMemcpyAsync(h->traj, u0, vb, cudaMemcpyDeviceToDevice, s));
        for (int n = 0; n < nsteps; ++n) {
            double* base = h->traj + (size_t)n * T.s * h->ndof;
            double* Y[4] = {base, base + h->ndof, base + 2 * h->ndof, base + 3 * h->ndof};
            double* next = n + 1 < nsteps ? h->traj + (size_t)(n + 1) * T.s * h->ndof : uT;
            SEM_TRY(rk_stages(h, T, dt, base, Y, next, s, count));
        }
    } else if (mode == SEM_CKPT_STATES) {
        SEM_CK(cudaMemcpyAsync(h->traj, u0, vb, cudaMemcpyDeviceToDevice, s));
        for (int n = 0; n < nsteps; ++n) {
            const double* un = h->traj + (size_t)n * h->ndof;
            double* next = n + 1 < nsteps ? h->traj + (size_t)(n + 1) * h->ndof : uT;
            SEM_TRY(rk_stages(h, T, dt, un, Yw, next, s, count));
        }
    } else {
        semh::CkptPlanner P(nsteps, slots);
        ckpt = P.forward_checkpoints(nsteps, slots);
        SEM_CK(cudaMemcpyAsync(h->traj, u0, vb, cudaMemcpyDeviceToDevice, s));
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
    h->have_fwd = true;
    h->f_scheme = scheme;
    h->f_nsteps = nsteps;
    h->f_dt = dt;
    h->f_mode = mode;
    h->f_slots = slots;
    h->f_ckpt = ckpt;
    h->st[0] = count;
    return SEM_OK;
}

int adjoint_impl(sem_t h, const double* lamT, double* lam0, cudaStream_t s) {
    if (!h->have_fwd) return fail(SEM_ERR_STATE, "sem_rk_adjoint needs a completed sem_rk_forward");
    SEM_TRY(check_state_ptr(lamT, "lamT"));
    SEM_TRY(check_state_ptr(lam0, "lam0"));
    if (lamT != lam0 && overlap(lamT, lam0, vec_bytes(h))) return fail(SEM_ERR_ALIAS, "lam0 partially overlaps lamT");
    Tableau T;
    tableau_of(h->f_scheme, T);
    const double dt = h->f_dt;
    const int nsteps = h->f_nsteps;
    const size_t vb = vec_bytes(h);
    if (lam0 != lamT) SEM_CK(cudaMemcpyAsync(lam0, lamT, vb, cudaMemcpyDeviceToDevice, s));
    {
        cudaError_t e = launch_scale(vec(h, V_NU), lam0, dt * T.b[T.s - 1], h->ndof, s);
        if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "scale launch: %s", cudaGetErrorString(e));
    }
    long long nrhs = 0, njt = 0;
    double* Yw[4] = {nullptr, vec(h, V_STAGE0), vec(h, V_STAGE0 + 1), vec(h, V_STAGE0 + 2)};
    if (h->f_mode == SEM_CKPT_STAGES) {
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
    h->st[1] = nrhs;
    h->st[2] = njt;
    return SEM_OK;
}

int objective_impl(sem_t h, const double* u, const double* uo, double* lam, cudaStream_t s) {
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
    cudaError_t e = launch_objective(u, uo, lam, h->partials, nb, a, s);
    if (e == cudaSuccess) e = launch_sum_partials(h->partials, nb, h->scal, 0.5, s);
    if (e != cudaSuccess) return fail(SEM_ERR_CUDA, "objective launch: %s", cudaGetErrorString(e));
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
    cudaFree(h->lvec);
    cudaFree(h->partials);
    cudaFree(h->scal);
    cudaFree(h->flag);
    cudaFree(h->vecs);
    cudaFree(h->traj);
    delete h;
}

size_t sem_ndof(sem_t h) { return h ? h->ndof : 0; }

int sem_coords(sem_t h, double* x) {
    if (!h || !x) return fail(SEM_ERR_ARG, "null handle or output");
    for (int g = 0; g < h->G; ++g) {
        const int e = g / h->N, i = g % h->N;
        x[g] = e * h->h + (h->xi[i] + 1.0) * h->h / 2.0;
    }
    return SEM_OK;
}

int sem_rhs(sem_t h, const double* u, double* f, void* stream) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    SEM_TRY(check_state_ptr(u, "u"));
    SEM_TRY(check_state_ptr(f, "f"));
    if (overlap(u, f, vec_bytes(h))) return fail(SEM_ERR_ALIAS, "f overlaps u");
    SEM_TRY(ensure_workspace(h));
    return apply(h, OP_RHS, u, nullptr, epi_plain(f, nullptr), (cudaStream_t)stream);
}

int sem_jac_apply(sem_t h, const double* u, const double* w, double* jw, void* stream) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    SEM_TRY(check_state_ptr(u, "u"));
    SEM_TRY(check_state_ptr(w, "w"));
    SEM_TRY(check_state_ptr(jw, "jw"));
    if (overlap(u, jw, vec_bytes(h)) || overlap(w, jw, vec_bytes(h))) return fail(SEM_ERR_ALIAS, "jw overlaps an input");
    SEM_TRY(ensure_workspace(h));
    return apply(h, OP_JAC, u, w, epi_plain(jw, nullptr), (cudaStream_t)stream);
}

int sem_jacT_apply(sem_t h, const double* u, const double* v, double* jtv, void* stream) {
    if (!h) return fail(SEM_ERR_ARG, "null handle");
    SEM_TRY(check_state_ptr(u, "u"));
    SEM_TRY(check_state_ptr(v, "v"));
    SEM_TRY(check_state_ptr(jtv, "jtv"));
    if (overlap(u, jtv, vec_bytes(h)) || overlap(v, jtv, vec_bytes(h))) return fail(SEM_ERR_ALIAS, "jtv overlaps an input");
    SEM_TRY(ensure_workspace(h));
    return apply(h, OP_JACT, u, v, epi_plain(jtv, nullptr), (cudaStream_t)stream);
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

int sem_objective_grad(sem_t h, int scheme, double dt, int nsteps, const double* u0, const double* uo,
                       double* J_host, double* grad, void* stream) {
    if (!h || !J_host) return fail(SEM_ERR_ARG, "null handle or J_host");
    SEM_TRY(check_state_ptr(uo, "u_obs"));
    SEM_TRY(check_state_ptr(grad, "grad"));
    if (overlap(grad, u0, vec_bytes(h)) || overlap(grad, uo, vec_bytes(h)))
        return fail(SEM_ERR_ALIAS, "grad overlaps an input");
    SEM_TRY(ensure_workspace(h));
    cudaStream_t s = (cudaStream_t)stream;
    double* uN = vec(h, V_UN);
    SEM_CK(cudaMemsetAsync(h->flag, 0, sizeof(unsigned), s));
    SEM_TRY(forward_impl(h, scheme, dt, nsteps, u0, uN, s));
    SEM_TRY(objective_impl(h, uN, uo, grad, s));
    SEM_TRY(adjoint_impl(h, grad, grad, s));
    unsigned f = 0;
    SEM_CK(cudaMemcpyAsync(J_host, h->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    SEM_CK(cudaMemcpyAsync(&f, h->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SEM_CK(cudaStreamSynchronize(s));
    if (f || !std::isfinite(*J_host)) return fail(SEM_ERR_NONFINITE, "non-finite values in the gradient evaluation");
    return SEM_OK;
}

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

int sem_profile(sem_t h, int every) {
    if (!h || every < 0) return fail(SEM_ERR_ARG, "null handle or negative sampling period");
    if (!every) SEM_TRY(prof_drain(h));
    h->prof = every;
    for (int i = 0; i < 4; ++i) h->prof_tick[i] = 0;
    return SEM_OK;
}

int sem_profile_read(sem_t h, double* ms4, long long* count4, int reset) {
    if (!h || !ms4 || !count4) return fail(SEM_ERR_ARG, "null handle or output");
    SEM_TRY(prof_drain(h));
    for (int i = 0; i < 4; ++i) {
        ms4[i] = h->prof_ms[i];
        count4[i] = h->prof_n[i];
        if (reset) {
            h->prof_ms[i] = 0;
            h->prof_n[i] = 0;
        }
    }
    return SEM_OK;
}

const char* sem_last_error(void) { return g_err.c_str(); }

}  // extern "C"

int semk::max_np(int D, bool fp32) { return (D == 3 && !fp32) ? 12 : 16; }

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
    v->mats = h->mats.data();
    return SEM_OK;
}

void semk::set_error(const char* msg) { g_err = msg; }
