// Tensor-core contractions for the 3D element kernels with n = 16 GLL points per
// direction (order N = 15), the one order of the workloads where an element tile is
// a sizeable dense contraction: along one direction, a 16 x 16 matrix applied to the
// 256 lines of a 16^3 tile is the product (256 x 16) . (16 x 16)^T (Sec. 3.3: the
// Kronecker factors of eqs. rhsvec / jactransvec applied as matrix-matrix products).
//
// Two forms, beside the even-odd CUDA-core kernels of op_elem_lean.cuh:
//
//  * FP32-bulk form on the 5th-generation tensor cores (tcgen05, TF32 inputs, FP32
//    accumulation in tensor memory).  TF32 keeps 11 significand bits, so each
//    operand is split into two TF32 parts, x = x_hi + x_lo (x_hi = tf32(x),
//    x_lo = tf32(x - x_hi)), and the product is accumulated as
//    X_lo B_hi + X_hi B_lo + X_hi B_hi (three products, near-FP32 accuracy; the
//    dropped X_lo B_lo term is below 2^-22 of |X||B|).  The line values are staged
//    in shared memory in the canonical K-major layout without swizzle (core
//    matrices of 8 rows x 16 bytes), one elected thread issues the MMAs, a commit
//    arrives on an mbarrier, and every thread reads its own line's results back from
//    tensor memory: with M = 128 rows per MMA, line t of the element lives in TMEM
//    lane t % 128, so thread t owns line t exactly as in the CUDA-core kernels and
//    the pointwise terms stay per thread.
//
//  * FP64 form on the DMMA path (mma.sync m8n8k4 f64: sm_100-family tensor cores
//    have no FP64 tcgen05 kind).  The fragments come straight from the padded tiles.
//
// Both keep the tile layout, the pass order and the summation order ((x + y) + z) of
// the lean kernels; only the 1D contractions change.
#pragma once
#include "op_elem_lean.cuh"

namespace semk {

// Full (not even-odd) element matrices of order 15 for the tensor-core kernels,
// row-major: A[out][in].
struct FullMats16 {
    double Dg[16][16];
    double Sv[16][16];
    double Gv[16][16];
    double Dd[16][16];
};

namespace tc {

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D[tmem] (+)= A[smem] . B[smem]^T, kind::tf32, one CTA
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on the mbarrier once every MMA this thread issued before has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive 32-bit columns of this thread's TMEM lane (warp w reads lanes 32 (w % 4) .. + 31)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    // the wait names the destination registers, so no use of them moves above it
    asm volatile(
        "tcgen05.wait::ld.sync.aligned;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
          "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
          "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
          "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
        :
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// ------------------------------------------------------------------ descriptors
// Shared-memory matrix descriptor, canonical K-major layout without swizzle: core
// matrices of 8 rows x 16 bytes stored as 128 contiguous bytes; lbo = byte distance
// between core matrices adjacent along K, sbo = between 8-row groups.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the sm_100 family; base offset 0, no swizzle
    return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row r, k) of a K = 16 TF32 operand in the canonical layout.
constexpr uint32_t LBO = 128;        // next 4 values along K
constexpr uint32_t SBO = 4 * 128;    // next 8 rows (K = 16 spans 4 core matrices)
__device__ __forceinline__ uint32_t kmaj_off(int r, int k) {
    return (uint32_t)((r >> 3) * SBO + (k >> 2) * LBO + (r & 7) * 16 + (k & 3) * 4);
}

// Bounded mbarrier wait: give up after WAIT_NS of GPU time (a pass takes microseconds).
constexpr unsigned long long WAIT_NS = 200ull * 1000 * 1000;
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace tc

// ================================================================== FP32-bulk, tcgen05
// Shared memory of the F kernel: U tiles (3), the partial tile, A (hi, lo) for 256
// rows x 16, B (hi, lo) for 32 rows x 16 (Dg then Sv), the mbarrier and the TMEM slot.
struct TcRhsSmem {
    static constexpr int S3 = Tile<16>::S3;
    static constexpr size_t tiles = 4 * (size_t)S3 * sizeof(float);
    static constexpr size_t a_bytes = 256 * 16 * 4;
    static constexpr size_t b_bytes = 32 * 16 * 4;
    static constexpr size_t a_hi = tiles, a_lo = a_hi + a_bytes, b_hi = a_lo + a_bytes, b_lo = b_hi + b_bytes;
    static constexpr size_t bar = b_lo + b_bytes, slot = bar + 8, total = slot + 8;
};

// Build the split B operand (rows: outputs of mat0 then mat1; K: inputs) from FP64 matrices.
__device__ __forceinline__ void tc_build_b(unsigned char* sm, size_t off_hi, size_t off_lo, const double (*m0)[16],
                                           const double (*m1)[16], int t) {
    for (int e = t; e < 32 * 16; e += blockDim.x) {
        const int n = e >> 4, k = e & 15;
        const double v = n < 16 ? m0[n][k] : m1[n - 16][k];
        const float hi = tc::tf32_rna((float)v);
        const float lo = tc::tf32_rna((float)(v - (double)hi));
        *reinterpret_cast<float*>(sm + off_hi + tc::kmaj_off(n, k)) = hi;
        *reinterpret_cast<float*>(sm + off_lo + tc::kmaj_off(n, k)) = lo;
    }
}

// Write line t (16 values) as row t of the split A operand.
__device__ __forceinline__ void tc_stage_row(unsigned char* sm, size_t off_hi, size_t off_lo, int t,
                                             const float (&x)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float4 h, l;
        float* hp = &h.x;
        float* lp = &l.x;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float v = x[4 * q + i];
            hp[i] = tc::tf32_rna(v);
            lp[i] = tc::tf32_rna(v - hp[i]);
        }
        *reinterpret_cast<float4*>(sm + off_hi + tc::kmaj_off(t, 4 * q)) = h;
        *reinterpret_cast<float4*>(sm + off_lo + tc::kmaj_off(t, 4 * q)) = l;
    }
}

// One elected thread: D[half h] = A_lo B_hi + A_hi B_lo + A_hi B_hi over K = 16 for both
// 128-row halves (12 MMAs, M = 128, N = 32), then a commit to the mbarrier.
__device__ __forceinline__ void tc_issue_3xtf32(unsigned char* sm, size_t a_hi, size_t a_lo, size_t b_hi, size_t b_lo,
                                                uint32_t tmem, uint64_t* bar) {
    constexpr uint32_t idesc = tc::idesc_tf32(128, 32);
    const uint32_t base = tc::smem_u32(sm);
    const size_t apart[3] = {a_lo, a_hi, a_hi};
    const size_t bpart[3] = {b_hi, b_lo, b_hi};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t acc = 0;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const uint64_t ad = tc::sdesc(base + (uint32_t)apart[p] + h * 16 * tc::SBO + ks * 2 * tc::LBO, tc::LBO,
                                              tc::SBO);
                const uint64_t bd = tc::sdesc(base + (uint32_t)bpart[p] + ks * 2 * tc::LBO, tc::LBO, tc::SBO);
                tc::mma_tf32(tmem + 32 * h, ad, bd, idesc, acc);
                acc = 1;
            }
        }
    }
    tc::mma_commit(bar);
}

// Bounded wait for the pass's MMAs; false if they did not complete within WAIT_NS.
// The result is made block-uniform by the caller (__syncthreads_and).
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
    const unsigned long long t0 = tc::now_ns();
    while (!tc::mbar_try_wait(bar, parity))
        if (tc::now_ns() - t0 > tc::WAIT_NS) return false;
    return true;
}

// F(u) element kernel, FP32-bulk form, n = 16, contractions on tcgen05 (one element per block).
__global__ void __launch_bounds__(256) rhs3_tc_kernel(const __grid_constant__ FullMats16 FM, const ElemArgs a,
                                                       unsigned* err) {
    using Tl = Tile<16>;
    using L = TcRhsSmem;
    constexpr int NP = 16, P = Tl::P, S2 = Tl::S2, S3 = Tl::S3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = threadIdx.x, w = t >> 5;
    const int e = blockIdx.x;
    float* sm = reinterpret_cast<float*>(smem_raw);
    float* sU[3] = {sm, sm + S3, sm + 2 * S3};
    float* sF = sm + 3 * S3;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + L::bar);
    uint32_t* slot = reinterpret_cast<uint32_t*>(smem_raw + L::slot);
    if (w == 0) {
        tc::tmem_alloc(slot, 64);
        tc::tmem_relinquish();
    }
    if (t == 32) {
        tc::mbar_init(bar, 1);
        tc::mbar_init_fence();
    }
    tc_build_b(smem_raw, L::b_hi, L::b_lo, FM.Dg, FM.Sv, t);
    pdl_wait();
    const int ex = e % a.E, ey = (e / a.E) % a.E, ez = e / (a.E * a.E);
    float rU[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) rU[c] = load3<float, NP>(sU[c], a.u, c, ex, ey, ez, t, true, a, false);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t my_tmem = tmem + ((uint32_t)(32 * (w & 3)) << 16) + 32 * (w >> 2);
    const int xb = t * P, yb = (t / NP) * S2 + t % NP, zb = (t / NP) * P + t % NP;
    float* out = reinterpret_cast<float*>(a.lvec) + (size_t)e * 3 * (NP * NP * NP) + (t / NP) * NP + t % NP;
    uint32_t parity = 0;
    bool ok = true;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
            const int base = d == 0 ? xb : (d == 1 ? yb : zb);
            const int stride = d == 0 ? 1 : (d == 1 ? P : S2);
            float x[NP];
#pragma unroll
            for (int m = 0; m < NP; ++m) x[m] = sU[c][base + m * stride];
            tc_stage_row(smem_raw, L::a_hi, L::a_lo, t, x);
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            // after a timed-out pass no further MMA is issued and every result is NaN
            if (ok) {
                if (t == 0) {
                    tc::fence_after_sync();
                    tc_issue_3xtf32(smem_raw, L::a_hi, L::a_lo, L::b_hi, L::b_lo, tmem, bar);
                }
                ok = __syncthreads_and(tc_wait(bar, parity)) != 0;
                parity ^= 1u;
            }
            tc::fence_after_sync();
            float v[32];
            tc::tmem_ld32(my_tmem, v);   // v[0..16): Dg x, v[16..32): Sv x
            if (!ok) {
#pragma unroll
                for (int m = 0; m < 32; ++m) v[m] = __int_as_float(0x7fc00000);
            }
            const float* sUd = sU[d];
            float r[NP];
#pragma unroll
            for (int m = 0; m < NP; ++m) r[m] = fmaf(-(rU[d] + sUd[base + m * stride]), v[m], v[16 + m]);
            if (d == 0) {
#pragma unroll
                for (int m = 0; m < NP; ++m) sF[base + m * stride] = r[m];
            } else if (d == 1) {
#pragma unroll
                for (int m = 0; m < NP; ++m) sF[base + m * stride] += r[m];
            } else {
#pragma unroll
                for (int m = 0; m < NP; ++m) out[(size_t)c * NP * NP * NP + m * NP * NP] = r[m] + sF[zb + m * S2];
            }
            tc::fence_before_sync();
        }
    }
    if (!ok) {
        // the MMAs of the timed-out pass may still be running: give them one more bounded
        // wait before the tensor memory is released
        if (t == 0 && err) atomicOr(err, 1u);
        tc_wait(bar, parity ^ 1u);
    }
    __syncthreads();
    if (w == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 64);
    }
}

// ================================================================== FP64, DMMA
// D (8 x 8) += A (8 x 4) . B (4 x 8), FP64 (mma.sync m8n8k4).
__device__ __forceinline__ void dmma_884(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

// F(u) element kernel, FP64 form, n = 16, contractions on the DMMA path.  Warp w owns
// lines 32 w .. 32 w + 31 of every pass, in four groups of 8 lines; lane (g, q) =
// (lane / 4, lane % 4) holds row g of a group's fragments and the outputs 2q, 2q + 1 of
// each 8-wide block of the 32 outputs (Dg then Sv).
__global__ void __launch_bounds__(256) rhs3_dmma_kernel(const __grid_constant__ FullMats16 FM, const ElemArgs a) {
    using Tl = Tile<16>;
    constexpr int NP = 16, P = Tl::P, S2 = Tl::S2, S3 = Tl::S3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31, g = lane >> 2, q = lane & 3;
    const int e = blockIdx.x;
    double* sm = reinterpret_cast<double*>(smem_raw);
    double* sU[3] = {sm, sm + S3, sm + 2 * S3};
    double* sF = sm + 3 * S3;
    // B fragments of Dg and Sv: b = Mat[n0 + g][k0 + q] for 4 k-steps x 2 n-blocks each
    double bDg[4][2], bSv[4][2];
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
#pragma unroll
        for (int nb = 0; nb < 2; ++nb) {
            bDg[ks][nb] = FM.Dg[8 * nb + g][4 * ks + q];
            bSv[ks][nb] = FM.Sv[8 * nb + g][4 * ks + q];
        }
    pdl_wait();
    const int ex = e % a.E, ey = (e / a.E) % a.E, ez = e / (a.E * a.E);
#pragma unroll
    for (int c = 0; c < 3; ++c) load3<double, NP>(sU[c], a.u, c, ex, ey, ez, t, true, a, false);
    __syncthreads();
    double* out = reinterpret_cast<double*>(a.lvec) + (size_t)e * 3 * (NP * NP * NP);
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
            const int stride = d == 0 ? 1 : (d == 1 ? P : S2);
#pragma unroll 1
            for (int grp = 0; grp < 4; ++grp) {
                const int line = 32 * w + 8 * grp + g;   // this lane's fragment row
                const int base = d == 0 ? line * P : (d == 1 ? (line / NP) * S2 + line % NP : (line / NP) * P + line % NP);
                double cg[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, cs[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const double av = sU[c][base + (4 * ks + q) * stride];
#pragma unroll
                    for (int nb = 0; nb < 2; ++nb) {
                        dmma_884(cg[nb][0], cg[nb][1], av, bDg[ks][nb]);
                        dmma_884(cs[nb][0], cs[nb][1], av, bSv[ks][nb]);
                    }
                }
#pragma unroll
                for (int nb = 0; nb < 2; ++nb)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int m = 8 * nb + 2 * q + h;   // output node along the line
                        const int id = base + m * stride;
                        const double r = fma(-sU[d][id], cg[nb][h], cs[nb][h]);
                        if (d == 0) sF[id] = r;
                        else if (d == 1) sF[id] += r;
                        else {
                            const int i = line % NP, j = line / NP;
                            out[(size_t)c * NP * NP * NP + m * NP * NP + j * NP + i] = r + sF[id];
                        }
                    }
            }
            __syncthreads();
        }
    }
}

}  // namespace semk
