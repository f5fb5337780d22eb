// sem_rhs_noalloc: F(u) without any device allocation.
//
// Some callers cannot call cudaMalloc at the point where they need F(u): code
// running inside a host application whose device memory is owned by its own
// pool or arena, real-time loops that must not take the implicit device-wide
// synchronisation a cudaMalloc/cudaFree can cause, or plug-ins that are not
// allowed to grow the process's device footprint after start-up.  For them
// this entry point evaluates the same operator as sem_rhs, but its only scratch
// (the element-local buffer between the element kernel and the gather-scatter
// sum) is a fixed file-scope device array instead of handle-owned memory.
//
// The array, SEM_NOALLOC_SCRATCH_BYTES bytes, is reserved on every GPU that
// loads libsem.so and stays there until the process exits.  Its device address
// is looked up once per device (the first call on each device does that set-up,
// with that device current); make the first call before any stream capture.
// All calls share the array and it keeps the last call's contents: nothing in
// it needs to start at zero (every valid entry is written before it is read),
// and calls whose kernels overlap on the GPU (different streams, or threads
// without ordering) race on it and must be serialised by the caller.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "sem.h"
#include "sem_internal.h"

namespace {

constexpr size_t SCRATCH_BYTES = SEM_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_ptr[MAX_DEVICES] = {nullptr};

int scratch_for_current_device(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        semk::set_error(cudaGetErrorString(e));
        return SEM_ERR_CUDA;
    }
    if (dev < 0 || dev >= MAX_DEVICES) {
        semk::set_error("sem_rhs_noalloc: device ordinal out of range");
        return SEM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            semk::set_error(e != cudaSuccess ? cudaGetErrorString(e) : "cudaGetSymbolAddress returned null");
            return SEM_ERR_CUDA;
        }
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return SEM_OK;
}

}  // namespace

extern "C" int sem_rhs_noalloc(sem_t h, const double* u, double* f, void* stream) {
    semk::HandleView v;
    if (semk::handle_view(h, &v) != SEM_OK) {
        semk::set_error("sem_rhs_noalloc: null handle");
        return SEM_ERR_ARG;
    }
    if (v.batch || !v.mats) {
        semk::set_error("sem_rhs_noalloc: handles of sem_batch_create are not supported (use sem_rhs)");
        return SEM_ERR_ARG;
    }
    if (!u || !f || ((uintptr_t)u % 8) || ((uintptr_t)f % 8)) {
        semk::set_error("sem_rhs_noalloc: u and f must be non-null and 8-byte aligned");
        return SEM_ERR_ARG;
    }
    const size_t bytes = v.ndof * sizeof(double);
    if ((const char*)u < (const char*)f + bytes && (const char*)f < (const char*)u + bytes) {
        semk::set_error("sem_rhs_noalloc: f overlaps u");
        return SEM_ERR_ALIAS;
    }
    const size_t need = v.lvec_elems * (v.fp32 ? sizeof(float) : sizeof(double));
    if (need > SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "sem_rhs_noalloc: this grid needs %zu bytes of element-local scratch; the allocation-free "
                 "entry point holds at most %zu bytes (use sem_rhs)", need, SCRATCH_BYTES);
        semk::set_error(msg);
        return SEM_ERR_ARG;
    }
    void* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != SEM_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    semk::ElemArgs a;
    a.u = u;
    a.w = nullptr;
    a.lvec = scratch;
    a.E = v.E;
    a.N = v.N;
    a.G = v.G;
    a.nelem = v.nelem;
    a.plane = (unsigned)v.ndof;
    a.in_f2 = 0;
    // the element kernel of the handle's precision, as sem_rhs runs it
    cudaError_t e;
    const int op = semk::OP_RHS;
    if (v.dfloat) {
        if (v.dim == 1) e = semk::launch_elem<semk::dfloat, 1>(v.np, op, v.mats, a, s);
        else if (v.dim == 2) e = semk::launch_elem<semk::dfloat, 2>(v.np, op, v.mats, a, s);
        else e = semk::launch_elem<semk::dfloat, 3>(v.np, op, v.mats, a, s);
    } else if (v.fp32) {
        if (v.dim == 1) e = semk::launch_elem<float, 1>(v.np, op, v.mats, a, s);
        else if (v.dim == 2) e = semk::launch_elem<float, 2>(v.np, op, v.mats, a, s);
        else e = semk::launch_elem<float, 3>(v.np, op, v.mats, a, s);
    } else {
        if (v.dim == 1) e = semk::launch_elem<double, 1>(v.np, op, v.mats, a, s);
        else if (v.dim == 2) e = semk::launch_elem<double, 2>(v.np, op, v.mats, a, s);
        else e = semk::launch_elem<double, 3>(v.np, op, v.mats, a, s);
    }
    if (e != cudaSuccess) {
        semk::set_error(cudaGetErrorString(e));
        return SEM_ERR_CUDA;
    }
    semk::AsmArgs aa;
    aa.D = v.dim;
    aa.E = v.E;
    aa.N = v.N;
    aa.G = v.G;
    aa.NP = v.np;
    aa.GD = (unsigned)(v.ndof / v.dim);
    aa.ndof = (unsigned)v.ndof;
    aa.scale_mult = 1;
    semk::Epi ep;
    memset(&ep, 0, sizeof(ep));
    ep.out[0] = f;
    ep.alpha[0] = 1.0;
    ep.nout = 1;
    e = semk::launch_assemble(v.fp32, scratch, aa, ep, s);
    if (e != cudaSuccess) {
        semk::set_error(cudaGetErrorString(e));
        return SEM_ERR_CUDA;
    }
    return SEM_OK;
}
