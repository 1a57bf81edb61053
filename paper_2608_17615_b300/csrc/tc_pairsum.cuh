// Batched pair sum on the 5th-generation tensor cores (tcgen05, kind::tf32).
//
// For R right-hand sides the naive part of the potential (the dense sum of
// Eq. linear_system_matrix, every source n != j) is
//     Y[j][r] = sum_s H0(k |x_j - x_s|) S_r[s],   S_r = w m f_r,
// a complex matrix product once the kernel matrix H is formed.  Written over
// the reals with K' = 2 x sources,
//     A[j][2s] = Re H, A[j][2s+1] = Im H,
//     B[r][2s] = Re S_r, B[r][2s+1] = -Im S_r        (column r: Re Y[j][r])
//     B[Rp+r][2s] = Im S_r, B[Rp+r][2s+1] = Re S_r   (column Rp+r: Im Y[j][r])
// so D = A B^T is one GEMM with M = 128 targets, N = 2 Rp columns.
//
// Accuracy.  A TF32 operand keeps 11 significant bits, so every operand is
// split, X = X_hi + X_lo with X_hi rounded to TF32, and three products
// A_hi B_hi + A_hi B_lo + A_lo B_hi are accumulated (the dropped A_lo B_lo and
// the TF32 truncation of the low parts leave ~2^-22 relative per product).
// The tensor core accumulates in FP32 in tensor memory; to keep the rounding
// of long sums out of the result the accumulator is restarted every F stages
// ("runs") and each run's total is folded into Kahan-compensated FP32 sums,
// which are also kept in tensor memory.  The chunk's result is written as an
// FP64 partial and the chunks are summed in FP64 by the apply epilogue.
//
// Work decomposition: a unit is (operator, tile of 128 targets, chunk of source
// stages); a persistent grid takes the units of all operators round-robin, so
// several scatterers of uneven size share one launch.  One stage = 16 sources = K' 32 =
// 4 MMA k-steps of K = 8 (x 3 split products).  Warp roles in a CTA:
//   warps 0..15  producers: expand the stage's densities into B_hi/B_lo and
//                form H for 128 targets x 16 sources into A_hi/A_lo
//                (FP32 table of H0 in t = r^2, double-float t), in shared memory;
//   warp 16      control: TMEM allocation; lane 0 issues the bulk copies (TMA)
//                of each stage's split densities and source coordinates and
//                the tcgen05.mma instructions;
//   warps 17..20 fold: restart/fold the run accumulators and write partials.
// Every wait is bounded (about one second); on expiry the CTA records an
// error code, stops issuing work, waits for what it already issued and exits.
#pragma once
#include <cstdint>

#define TC_M 128
#define TC_SRC 16
#define TC_NS 2
#define TC_NSTG_MAX 3
#define TC_PROD_WARPS 16
#define TC_CTRL_WARP 16
#define TC_FOLD_WARP0 17
#define TC_THREADS (21 * 32)
#define TC_WAIT_NS 1000000000ull
#define TC_MAX_OPS 64

// One operator (scatterer) of a launch.  Units of all operators are numbered
// consecutively: operator s owns units [unit_begin, unit_begin + units).
struct TCOp {
    const float4* xy32;   // [npad] double-float node coordinates (x_hi, x_lo, y_hi, y_lo)
    const float4* Sc;     // [npad][Rp] split densities (re_hi, re_lo, im_hi, im_lo)
    const float4* tab;    // FP32 H0 table (k_pairsum_multi_f32 layout)
    double2* partial;     // [R][part_nchunk][n] FP64 chunk partials
    double k, inv_k;
    int n, tblocks, spc, nchunk, part_nchunk, unit_begin, units;
    int ncell, noct, b_lo, tab_words;
};

struct TCArgs {
    const TCOp* ops;      // [S] in device memory
    int S, total_units;
    int R, Rp, N, F;      // right-hand sides of this launch, padded count, GEMM columns 2 Rp, run length
    int nstg;             // staging slots (2 or 3)
    int r_offset;         // first right-hand side of this launch in the partial layout
    uint32_t idesc;
    int* err;             // device error word (0 = ok)
    uint64_t stall_ns;    // failure-detection test: > 0 makes the MMA issuer wait this long on a
                          // barrier that nothing completes, then abort like a stalled pipeline
};

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = TC_WAIT_NS) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (now_ns() - t0 > limit_ns) return false;
    }
}

// As mbar_wait, but also gives up (false) as soon as another role of the CTA has
// raised the abort flag, so that one stalled wait ends the whole pipeline quickly.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, const int* abort_flag) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = now_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*(const volatile int*)abort_flag) return false;
        if (now_ns() - t0 > TC_WAIT_NS) return false;
    }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor, no swizzle: 8-row x 16-byte core matrices,
// lbo = byte distance between core matrices along K, sbo = along M/N.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 lanes x 16 columns of 32 bits: thread t gets lane (taddr.lane + t), columns col .. col + 15.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}

// Round to the nearest TF32 value (ties away from zero); the remainder x - tf32(x) is exact in FP32.
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u); }

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

}  // namespace tc

__device__ __noinline__ float2 tc_h0_direct(double t, double k, double inv_k) {
    double2 h = ls_h0_r2(t, k, inv_k);
    return make_float2((float)h.x, (float)h.y);
}

// S_r[s] = w_s m_s f_r[s] split into TF32 high parts and FP32 remainders; zero beyond n or R.
__global__ void k_tc_prep_S(int n, int npad, int R, int Rp, const double2* __restrict__ f, size_t sf,
                            const double* __restrict__ w, const double2* __restrict__ m, float4* __restrict__ Sc) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)npad * Rp) return;
    const int r = (int)(idx / npad), s = (int)(idx % npad);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s < n && r < R) {
        double2 ff = f[(size_t)r * sf + s];
        if (m) {
            double2 mm = m[s];
            ff = make_double2(mm.x * ff.x - mm.y * ff.y, mm.x * ff.y + mm.y * ff.x);
        }
        const double ww = w ? w[s] : 1.0;
        const double re = ww * ff.x, im = ww * ff.y;
        const float rh = tc::tf32_hi((float)re), ih = tc::tf32_hi((float)im);
        v = make_float4(rh, (float)(re - (double)rh), ih, (float)(im - (double)ih));
    }
    Sc[(size_t)s * Rp + r] = v;
}

// Node coordinates as double-float pairs, zero-padded to npad.
__global__ void k_tc_xy32(int n, int npad, const double2* __restrict__ xy, float4* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < n) {
        double2 p = xy[i];
        float xh = (float)p.x, yh = (float)p.y;
        v = make_float4(xh, (float)(p.x - (double)xh), yh, (float)(p.y - (double)yh));
    }
    out[i] = v;
}

struct TCShared {
    uint64_t full[TC_NS], empty[TC_NS], stfull[TC_NSTG_MAX], stempty[TC_NSTG_MAX], accfull[2], accempty[2], done, tabbar;
    uint64_t never;       // initialised, never arrived on (failure-detection test only)
    uint32_t tmem;
    int abort_flag;
};

// Unit cursor shared by all roles: global unit u (operator s, target tile, source chunk),
// local stage g of G.
struct TCCursor {
    int u, s, g, G, tile, chunk, s_begin, s_end;
    __device__ void start(const TCArgs& a) {
        u = blockIdx.x;
        g = 0;
        load(a);
    }
    __device__ void load(const TCArgs& a) {
        if (u >= a.total_units) return;
        s = 0;
        while (s + 1 < a.S && a.ops[s + 1].unit_begin <= u) ++s;
        const TCOp& o = a.ops[s];
        const int lu = u - o.unit_begin;
        tile = lu % o.tblocks;
        chunk = lu / o.tblocks;
        s_begin = chunk * o.spc;
        s_end = min(o.n, s_begin + o.spc);
        G = (s_end - s_begin + TC_SRC - 1) / TC_SRC;
    }
    __device__ bool valid(const TCArgs& a) const { return u < a.total_units; }
    __device__ void next(const TCArgs& a) {
        if (++g >= G) {
            g = 0;
            u += gridDim.x;
            load(a);
        }
    }
};

__global__ void __launch_bounds__(TC_THREADS, 1) k_pairsum_tc(TCArgs a) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ TCShared sh;
    // dynamic shared memory: ring of TC_NS stages {A_hi, A_lo, B_hi, B_lo}, nstg staging slots
    // {Sc tile, coordinates}, then the H0 table of the current operator (the largest fits)
    unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    const int N = a.N, Rp = a.Rp;
    const uint32_t a_bytes = TC_M * 2 * TC_SRC * 4;            // 16 KB
    const uint32_t b_bytes = (uint32_t)N * 2 * TC_SRC * 4;     // 8 KB at N = 64
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    const uint32_t sc_bytes = (uint32_t)TC_SRC * Rp * 16;
    const uint32_t xy_bytes = TC_SRC * 16;
    const uint32_t stg_bytes = sc_bytes + xy_bytes;
    unsigned char* ring = base;
    unsigned char* stg = ring + TC_NS * stage_bytes;
    const uint32_t nstg = (uint32_t)a.nstg;
    float4* ftab = (float4*)(stg + nstg * stg_bytes);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_NS; ++s) {
            tc::mbar_init(&sh.full[s], TC_PROD_WARPS);
            tc::mbar_init(&sh.empty[s], 1);
        }
        for (int s = 0; s < TC_NSTG_MAX; ++s) {
            tc::mbar_init(&sh.stfull[s], 1);
            tc::mbar_init(&sh.stempty[s], TC_PROD_WARPS);
        }
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&sh.accfull[s], 1);
            tc::mbar_init(&sh.accempty[s], 4);
        }
        tc::mbar_init(&sh.done, 1);
        tc::mbar_init(&sh.tabbar, TC_PROD_WARPS);
        tc::mbar_init(&sh.never, 1);
        sh.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const uint32_t tmem_cols = 4u * (uint32_t)N;
    if (warp == TC_CTRL_WARP) {
        tc::tmem_alloc(&sh.tmem, tmem_cols);
        tc::fence_before();
    }
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = sh.tmem;

    if (warp < TC_PROD_WARPS) {
        // ---------------------------------------------------------------- producers
        const int p = threadIdx.x;
        const int row = p & (TC_M - 1), q = p >> 7;
        TCCursor c;
        c.start(a);
        int cur_unit = -1, cur_op = -1;
        float txh = 0.f, txl = 0.f, tyh = 0.f, tyl = 0.f;
        const float2* coef = nullptr;
        const float4* cellv = nullptr;
        const int2* oct = nullptr;
        int noct = 0, b_lo = 0;
        double kk = 1.0, inv_k = 1.0;
        uint32_t tab_phase = 0;
        auto prod_sync = [&]() -> bool {
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sh.tabbar);
            const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&sh.tabbar, tab_phase & 1));
            ++tab_phase;
            return ok;
        };
        for (uint32_t gs = 0; c.valid(a); ++gs, c.next(a)) {
            if (c.s != cur_op) {
                // the operator changed: once every producer is past its previous stage, reload
                // the table (bounded mbarrier syncs among the producer warps, not bar.sync,
                // so that a producer that gave up cannot leave the others waiting forever)
                const TCOp& o = a.ops[c.s];
                bool ok = prod_sync();
                if (ok) {
                    for (int i = p; i < o.tab_words; i += TC_PROD_WARPS * 32) ftab[i] = o.tab[i];
                    ok = prod_sync();
                }
                if (!ok) {
                    if (lane == 0) { atomicOr(a.err, 32); sh.abort_flag = 1; }
                    break;
                }
                const int coef_f4 = (o.ncell * NC_F32 + 1) / 2;
                coef = reinterpret_cast<const float2*>(ftab);
                cellv = ftab + coef_f4;
                oct = reinterpret_cast<const int2*>(cellv + o.ncell);
                noct = o.noct;
                b_lo = o.b_lo;
                kk = o.k;
                inv_k = o.inv_k;
                cur_op = c.s;
            }
            if (c.u != cur_unit) {
                cur_unit = c.u;
                const TCOp& o = a.ops[c.s];
                const int j = c.tile * TC_M + row;
                float4 t = o.xy32[min(j, o.n - 1)];
                txh = t.x; txl = t.y; tyh = t.z; tyl = t.w;
            }
            const uint32_t slot = gs % TC_NS, stgi = gs % nstg;
            // 1. the staged densities and coordinates of this stage: form H (and read this
            //    thread's B operands) while the MMAs of earlier stages still hold the ring slot
            bool ok = tc::mbar_wait_or_abort(&sh.stfull[stgi], (gs / nstg) & 1, &sh.abort_flag);
            ok = __all_sync(0xffffffffu, ok);                 // one decision per warp
            if (!ok) {
                if (lane == 0) { atomicOr(a.err, 1); sh.abort_flag = 1; }
                break;
            }
            if (__any_sync(0xffffffffu, *(volatile int*)&sh.abort_flag)) break;
            const float4* sc = (const float4*)(stg + stgi * stg_bytes);
            const float4* sxy = (const float4*)(stg + stgi * stg_bytes + sc_bytes);
            // B: K-element pair c2 = sources (2 c2, 2 c2 + 1); element (col, kk) at float4 (kk / 4) * N + col;
            // 8 Rp <= 512 items, at most one per producer thread
            const bool has_b = p < 8 * Rp;
            float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
            int b_c2 = 0, b_r = 0;
            if (has_b) {
                b_c2 = p / Rp;
                b_r = p - b_c2 * Rp;
                v0 = sc[(2 * b_c2) * Rp + b_r];
                v1 = sc[(2 * b_c2 + 1) * Rp + b_r];
            }
            // A: sources 4q .. 4q + 3 of the stage for target j; element (row, kk) at float4 (kk / 4) * 128 + row
            float hr[4], hi[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int sl = 4 * q + e;
                const int src = c.s_begin + c.g * TC_SRC + sl;
                hr[e] = 0.f;
                hi[e] = 0.f;
                if (src >= c.s_end) continue;
                const float4 sc4 = sxy[sl];
                float dxh, dxl, dyh, dyl;
                df_diff(txh, txl, sc4.x, sc4.y, dxh, dxl);
                df_diff(tyh, tyl, sc4.z, sc4.w, dyh, dyl);
                float p1 = dxh * dxh, e1 = fmaf(dxh, dxh, -p1);
                e1 = fmaf(2.f * dxh, dxl, e1);
                float p2 = dyh * dyh, e2 = fmaf(dyh, dyh, -p2);
                e2 = fmaf(2.f * dyh, dyl, e2);
                float th, tl;
                two_sum(p1, p2, th, tl);
                tl += e1 + e2;
                float t0 = th + tl;
                tl = tl - (t0 - th);
                th = t0;
                const int bits = __float_as_int(th);
                const unsigned o = (unsigned)((bits >> 23) - b_lo);
                if (o < (unsigned)noct) {
                    const int2 ob = oct[o];
                    const int cell = ob.x + ((bits & 0x7fffff) >> ob.y);
                    const float4 cv = cellv[cell];
                    const float u = ((th - cv.x) + (tl - cv.y)) * cv.z;
                    const float2* cc = coef + cell * NC_F32;
                    float2 k2 = cc[NC_F32 - 1];
                    float vr = k2.x, vi = k2.y;
#pragma unroll
                    for (int d = NC_F32 - 2; d >= 0; --d) {
                        k2 = cc[d];
                        vr = fmaf(vr, u, k2.x);
                        vi = fmaf(vi, u, k2.y);
                    }
                    hr[e] = vr;
                    hi[e] = vi;
                } else if (th > 0.f) {
                    const float2 h = tc_h0_direct((double)th + (double)tl, kk, inv_k);
                    hr[e] = h.x;
                    hi[e] = h.y;
                }
                // th == 0: the self pair, excluded from the naive sum
            }
            // the staging slot has been read (densities and coordinates): free for the next copy
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sh.stempty[stgi]);
            // 2. the ring slot: wait for the MMAs of stage gs - TC_NS, then store the operands
            if (gs >= TC_NS) ok = tc::mbar_wait_or_abort(&sh.empty[slot], ((gs / TC_NS) - 1) & 1, &sh.abort_flag);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) { atomicOr(a.err, 1); sh.abort_flag = 1; }
                break;
            }
            if (__any_sync(0xffffffffu, *(volatile int*)&sh.abort_flag)) break;
            unsigned char* st = ring + slot * stage_bytes;
            float4* Ahi = (float4*)st;
            float4* Alo = (float4*)(st + a_bytes);
            float4* Bhi = (float4*)(st + 2 * a_bytes);
            float4* Blo = (float4*)(st + 2 * a_bytes + b_bytes);
            if (has_b) {
                Bhi[b_c2 * N + b_r] = make_float4(v0.x, -v0.z, v1.x, -v1.z);
                Bhi[b_c2 * N + Rp + b_r] = make_float4(v0.z, v0.x, v1.z, v1.x);
                Blo[b_c2 * N + b_r] = make_float4(v0.y, -v0.w, v1.y, -v1.w);
                Blo[b_c2 * N + Rp + b_r] = make_float4(v0.w, v0.y, v1.w, v1.y);
            }
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const float x0 = hr[2 * h2], y0 = hi[2 * h2], x1 = hr[2 * h2 + 1], y1 = hi[2 * h2 + 1];
                const float x0h = tc::tf32_hi(x0), y0h = tc::tf32_hi(y0), x1h = tc::tf32_hi(x1), y1h = tc::tf32_hi(y1);
                Ahi[(2 * q + h2) * TC_M + row] = make_float4(x0h, y0h, x1h, y1h);
                Alo[(2 * q + h2) * TC_M + row] = make_float4(x0 - x0h, y0 - y0h, x1 - x1h, y1 - y1h);
            }
            tc::fence_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sh.full[slot]);
        }
    } else if (warp == TC_CTRL_WARP) {
        // ---------------------------------------------------------------- control (one thread)
        if (lane == 0) {
            TCCursor c, cs;
            c.start(a);
            cs.start(a);
            uint32_t issued = 0;          // staging copies issued (stage index order)
            auto issue_stage = [&](uint32_t gsi) {
                const uint32_t si = gsi % nstg;
                unsigned char* dst = stg + si * stg_bytes;
                const int sbase = cs.s_begin + cs.g * TC_SRC;
                const TCOp& o = a.ops[cs.s];
                tc::mbar_expect_tx(&sh.stfull[si], stg_bytes);
                tc::bulk_g2s(dst, o.Sc + (size_t)sbase * Rp, sc_bytes, &sh.stfull[si]);
                tc::bulk_g2s(dst + sc_bytes, o.xy32 + sbase, xy_bytes, &sh.stfull[si]);
                cs.next(a);
            };
            for (; issued < nstg && cs.valid(a); ++issued) issue_stage(issued);
            const uint32_t lbo_a = TC_M * 16, lbo_b = (uint32_t)N * 16, sbo = 128;
            const uint32_t ring_addr = tc::smem_u32(ring);
            uint32_t rr = 0;              // runs started
            bool ok = true;
            if (a.stall_ns && !tc::mbar_wait(&sh.never, 0, a.stall_ns)) {
                atomicOr(a.err, 64);
                sh.abort_flag = 1;
                ok = false;
            }
            for (uint32_t gs = 0; ok && c.valid(a); ++gs, c.next(a)) {
                const uint32_t slot = gs % TC_NS;
                const bool first = (c.g % a.F) == 0;
                const bool last = ((c.g % a.F) == a.F - 1) || (c.g == c.G - 1);
                const uint32_t ab = rr & 1;
                // once the producers have read staging slot gs % nstg, refill it with stage gs + nstg
                if (issued == gs + nstg && cs.valid(a)) {
                    ok = tc::mbar_wait_or_abort(&sh.stempty[gs % nstg], (gs / nstg) & 1, &sh.abort_flag);
                    if (ok) {
                        issue_stage(issued);
                        ++issued;
                    }
                }
                if (ok && first && rr >= 2) ok = tc::mbar_wait_or_abort(&sh.accempty[ab], ((rr >> 1) - 1) & 1, &sh.abort_flag);
                if (ok) ok = tc::mbar_wait_or_abort(&sh.full[slot], (gs / TC_NS) & 1, &sh.abort_flag);
                if (!ok || *(volatile int*)&sh.abort_flag) {
                    if (!ok) { atomicOr(a.err, 2); sh.abort_flag = 1; }
                    break;
                }
                tc::fence_after();
                const uint32_t sa = ring_addr + slot * stage_bytes;
                const uint32_t a_hi = sa, a_lo = sa + a_bytes, b_hi = sa + 2 * a_bytes, b_lo = b_hi + b_bytes;
                const uint32_t d = tmem + ab * (uint32_t)N;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint32_t oa = ks * 2 * TC_M * 16, ob = ks * 2 * (uint32_t)N * 16;
                    const uint64_t dah = tc::sdesc(a_hi + oa, lbo_a, sbo), dal = tc::sdesc(a_lo + oa, lbo_a, sbo);
                    const uint64_t dbh = tc::sdesc(b_hi + ob, lbo_b, sbo), dbl = tc::sdesc(b_lo + ob, lbo_b, sbo);
                    tc::mma_tf32(d, dah, dbh, a.idesc, (first && ks == 0) ? 0u : 1u);
                    tc::mma_tf32(d, dah, dbl, a.idesc, 1u);
                    tc::mma_tf32(d, dal, dbh, a.idesc, 1u);
                }
                tc::mma_commit(&sh.empty[slot]);
                if (last) {
                    tc::mma_commit(&sh.accfull[ab]);
                    ++rr;
                }
            }
            // drain: every issued MMA and bulk copy completes before the CTA exits (after an
            // abort the last nstg copies may not have been consumed; waiting on a completed
            // phase returns at once)
            tc::mma_commit(&sh.done);
            if (!tc::mbar_wait(&sh.done, 0)) atomicOr(a.err, 4);
            for (uint32_t gsi = (issued >= nstg ? issued - nstg : 0); gsi < issued; ++gsi)
                if (!tc::mbar_wait(&sh.stfull[gsi % nstg], (gsi / nstg) & 1)) atomicOr(a.err, 16);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- fold warps
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        const uint32_t col_sum = 2u * N, col_cmp = 3u * N;
        TCCursor c;
        c.start(a);
        uint32_t rr = 0;
        while (c.valid(a)) {
            const int nruns = (c.G + a.F - 1) / a.F;
            bool ok = true;
            for (int kr = 0; kr < nruns; ++kr, ++rr) {
                const uint32_t ab = rr & 1;
                ok = __all_sync(0xffffffffu, tc::mbar_wait_or_abort(&sh.accfull[ab], (rr >> 1) & 1, &sh.abort_flag));
                if (!ok) {
                    if (lane == 0) { atomicOr(a.err, 8); sh.abort_flag = 1; }
                    break;
                }
                if (__any_sync(0xffffffffu, *(volatile int*)&sh.abort_flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                for (int c0 = 0; c0 < N; c0 += 16) {
                    float acc[16], s[16], cp[16];
                    tc::tmem_ld16(tl + ab * (uint32_t)N + c0, acc);
                    if (kr == 0) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) { s[i] = acc[i]; cp[i] = 0.f; }
                    } else {
                        tc::tmem_ld16(tl + col_sum + c0, s);
                        tc::tmem_ld16(tl + col_cmp + c0, cp);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const float y = acc[i] - cp[i];
                            const float t = s[i] + y;
                            cp[i] = (t - s[i]) - y;
                            s[i] = t;
                        }
                    }
                    tc::tmem_st16(tl + col_sum + c0, s);
                    tc::tmem_st16(tl + col_cmp + c0, cp);
                }
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&sh.accempty[ab]);
            }
            if (!ok) break;
            // the unit's result: Re at columns r, Im at columns Rp + r
            const TCOp& o = a.ops[c.s];
            const int j = c.tile * TC_M + row;
            for (int r0 = 0; r0 < Rp; r0 += 16) {
                float sr[16], cr[16], si[16], ci[16];
                tc::tmem_ld16(tl + col_sum + r0, sr);
                tc::tmem_ld16(tl + col_cmp + r0, cr);
                tc::tmem_ld16(tl + col_sum + Rp + r0, si);
                tc::tmem_ld16(tl + col_cmp + Rp + r0, ci);
                if (j < o.n) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int r = r0 + i;
                        if (r < a.R)
                            o.partial[((size_t)(a.r_offset + r) * o.part_nchunk + c.chunk) * o.n + j] =
                                make_double2((double)sr[i] - (double)cr[i], (double)si[i] - (double)ci[i]);
                    }
                }
            }
            // jump to the next unit
            c.g = c.G - 1;
            c.next(a);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == TC_CTRL_WARP) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, tmem_cols);
    }
}

// Self-check of the tensor-core path: D = A B^T for one 128 x N x 32 tile of
// exactly representable values through the same layouts, descriptors and MMA
// sequence (hi parts only), written as D[row][col] to out.
__global__ void __launch_bounds__(128, 1) k_tc_gemm_check(const float* __restrict__ A, const float* __restrict__ B, int N,
                                                          float* __restrict__ out, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tm;
    unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    float4* As = (float4*)base;
    float4* Bs = (float4*)(base + TC_M * 32 * 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // A [128][32], B [N][32] row-major in global; element (row, kk) at float4 (kk / 4) * rows + row
    for (int i = threadIdx.x; i < TC_M * 8; i += blockDim.x) {
        const int row = i % TC_M, c4 = i / TC_M;
        As[c4 * TC_M + row] = *reinterpret_cast<const float4*>(A + row * 32 + 4 * c4);
    }
    for (int i = threadIdx.x; i < N * 8; i += blockDim.x) {
        const int row = i % N, c4 = i / N;
        Bs[c4 * N + row] = *reinterpret_cast<const float4*>(B + row * 32 + 4 * c4);
    }
    tc::fence_async_smem();
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t ncols = 32;                        // a power of two >= N
    while (ncols < (uint32_t)N) ncols *= 2;
    if (warp == 0) {
        tc::tmem_alloc(&tm, ncols);
        tc::fence_before();
    }
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tm;
    if (threadIdx.x == 0) {
        const uint32_t sa = tc::smem_u32(As), sb = tc::smem_u32(Bs);
        const uint32_t idesc = tc::idesc_tf32(TC_M, N);
        for (int ks = 0; ks < 4; ++ks) {
            const uint64_t da = tc::sdesc(sa + ks * 2 * TC_M * 16, TC_M * 16, 128);
            const uint64_t db = tc::sdesc(sb + ks * 2 * N * 16, N * 16, 128);
            tc::mma_tf32(tmem, da, db, idesc, ks > 0 ? 1u : 0u);
        }
        tc::mma_commit(&bar);
    }
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&bar, 0));
    if (!ok && lane == 0) atomicOr(err, 1);
    tc::fence_after();
    if (ok) {
        const int row = warp * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tl + c0, v);
            for (int i = 0; i < 16; ++i) out[row * N + c0 + i] = v[i];
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, ncols);
    }
}
