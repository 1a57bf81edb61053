// B300 (sm_103a) implementation of the Lippmann-Schwinger Nystrom hot path
// behind the C ABI of include/lsgpu.h.
//
// Kernels (all FP64, complex as double2):
//   k_pairsum        dense pair sum sum_{n != j} H0(k |y_j - y_n|) s_n, sources staged
//                    through shared memory, one target per thread, the source range
//                    split into chunks whose partial sums land in a scratch buffer
//   k_apply_epi      warp per row: sums the chunk partials in a fixed order, the CSR
//                    correction (VDIM dV, Eq. DIM_decomp) and the epilogue
//                    (L x)_j = x_j + k^2 [(i/4) sum + sum_q dV_jq m_q x_q]  (Eq. linear_system_matrix)
//   k_tqc            T_Q^C gather (Approach II, Eq. T_H^C_def) over the transposed CSR
//   k_stencil        t = A g with the 3 x 3 sparsifying stencils (Eq. sparsifying_min), one per
//                    grid-row class (interior, edges, corners; Eq. cart_neighbors_LS)
//   k_cr_mv/k_cr_tri block-cyclic-reduction solve C t' = t (Eq. LC_def): batched dense
//                    block products per level (cr_solve.cuh); the batched forms use the
//                    block LU sweeps k_bt_fwd_multi / k_bt_bwd_multi
//   k_tcq            z_q = w_q + sum_4 psi (t' - g) (Eq. preconditioner_factored)
//   k_dots/k_sumrows/k_update/k_norm...  classical Gram-Schmidt (twice) for GMRES
//   k_givens         Hessenberg column update and Givens rotation, residual history
//   k_farfield       u_inf(theta) = -k^2 e^{i pi/4}/sqrt(8 pi k) sum_j w_j m_j u_j e^{-i k xhat . y_j}
//   k_incident       b_j = exp(i k d . y_j)
//   k_pairsum_tc     batched pair sum as a tcgen05 (kind::tf32) GEMM, tc_pairsum.cuh
// Device H0^(1): ascending series of J0, Y0 for z <= 6 (Abramowitz & Stegun 9.1.12,
// 9.1.13); for z > 6 the modulus/phase form sqrt(2/(pi z)) (P + i Q) e^{i(z - pi/4)}
// with P, zQ fitted polynomials in 36/z^2 (constants in hankel_fit.h).
#include <cuda_runtime.h>
#include <cublas_v2.h>
#include <cufft.h>
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lsgpu.h"
#include "hankel_fit.h"
#include "ls_internal.h"

using lsgpu::CsrC;
using lsgpu::GridSetup;
using lsgpu::HostMesh;

static thread_local std::string g_err;

static ls_status fail(ls_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(LS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

#define CKS(call)                                                                                 \
    do {                                                                                          \
        cusolverStatus_t s_ = (call);                                                             \
        if (s_ != CUSOLVER_STATUS_SUCCESS)                                                        \
            return fail(LS_ECUDA, std::string(#call) + ": cusolver status " + std::to_string(s_)); \
    } while (0)

#define TRY(x)                         \
    do {                               \
        ls_status s__ = (x);           \
        if (s__ != LS_OK) return s__;  \
    } while (0)

// The dynamic shared-memory limit is a per-kernel attribute shared by all operators:
// only ever raise it, so that an operator with a smaller table cannot invalidate
// another operator's launches.
template <typename K>
static cudaError_t raise_smem_limit(K kernel, size_t bytes) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    if ((size_t)a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 conjmul(double2 a, double2 b) {   // conj(a) * b
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sparsifying stencils (Eq. sparsifying_min) per grid-row class c = ca + 3 cb (ca = 0 on the
// first column, 1 inside, 2 on the last; cb likewise): st[9 c + (da+1) + 3 (db+1)], zero at
// offsets that leave the grid (Eq. cart_neighbors_LS truncates the neighbourhood to D).
__device__ __forceinline__ int grid_row_class(int a, int b, int nx, int ny) {
    const int ca = a == 0 ? 0 : (a == nx - 1 ? 2 : 1);
    const int cb = b == 0 ? 0 : (b == ny - 1 ? 2 : 1);
    return ca + 3 * cb;
}

#define LS_INV_SQRT_PI 0.56418958354775628695
#define LS_TWO_OVER_PI 0.63661977236758134308
#define LS_EULER_GAMMA 0.57721566490153286061

// H0^(1)(z) for z = k r given r^2 > 0.
__device__ __forceinline__ double2 ls_h0_r2(double r2, double k, double inv_k) {
    double ir = rsqrt(r2);
    double r = r2 * ir;
    double z = k * r;
    if (z > LS_H0_ZSPLIT) {
        double iz = ir * inv_k;
        double s = 36.0 * iz * iz;
        double P = ls_h0_p[LS_H0_DEG], Qz = ls_h0_qz[LS_H0_DEG];
#pragma unroll
        for (int i = LS_H0_DEG - 1; i >= 0; --i) {
            P = fma(P, s, ls_h0_p[i]);
            Qz = fma(Qz, s, ls_h0_qz[i]);
        }
        double Q = Qz * iz;
        double sz, cz;
        sincos(z, &sz, &cz);
        double amp = LS_INV_SQRT_PI * rsqrt(z);
        double c1 = cz + sz, s1 = sz - cz;     // sqrt(2) cos(z - pi/4), sqrt(2) sin(z - pi/4)
        return make_double2(amp * fma(P, c1, -Q * s1), amp * fma(P, s1, Q * c1));
    }
    double q = 0.25 * z * z;
    double t = 1.0, j0 = 1.0, S = 0.0;
#pragma unroll 4
    for (int i = 0; i < LS_H0_NSERIES; ++i) {
        t *= -q * ls_h0_rk2[i];
        j0 += t;
        S = fma(-ls_h0_hk[i], t, S);
    }
    double y0 = LS_TWO_OVER_PI * fma(log(0.5 * z) + LS_EULER_GAMMA, j0, S);
    return make_double2(j0, y0);
}

// ------------------------------------------------------------------ pair sum
#define PS_TPB 128
#define PS_TILE 256

// partial[c][j] = sum_{n in chunk c, n != j} H0(k |y_j - y_n|) s_n,  s_n = w_n (m_n) f_n
__global__ void __launch_bounds__(PS_TPB) k_pairsum(const double2* __restrict__ xy, const double* __restrict__ w,
                                                    const double2* __restrict__ m, const double2* __restrict__ f,
                                                    int n, int src_per_chunk, double k, double inv_k,
                                                    double2* __restrict__ partial) {
    __shared__ double4 tile[PS_TILE];
    const int j = blockIdx.x * PS_TPB + threadIdx.x;
    const int s_begin = blockIdx.y * src_per_chunk;
    const int s_end = min(n, s_begin + src_per_chunk);
    const double2 yj = xy[min(j, n - 1)];
    double ar = 0.0, ai = 0.0;
    for (int base = s_begin; base < s_end; base += PS_TILE) {
        __syncthreads();
        for (int i = threadIdx.x; i < PS_TILE; i += PS_TPB) {
            int src = base + i;
            double4 v = make_double4(0.0, 0.0, 0.0, 0.0);
            if (src < s_end) {
                double2 p = xy[src];
                double2 ff = f[src];
                if (m) ff = cmul(m[src], ff);
                double ww = w ? w[src] : 1.0;
                v = make_double4(p.x, p.y, ww * ff.x, ww * ff.y);
            }
            tile[i] = v;
        }
        __syncthreads();
        const int cnt = min(PS_TILE, s_end - base);
        for (int i = 0; i < cnt; ++i) {
            double4 s = tile[i];
            double dx = yj.x - s.x, dy = yj.y - s.y;
            double r2 = fma(dx, dx, dy * dy);
            if (r2 > 0.0) {
                double2 h = ls_h0_r2(r2, k, inv_k);
                ar = fma(h.x, s.z, fma(-h.y, s.w, ar));
                ai = fma(h.x, s.w, fma(h.y, s.z, ai));
            }
        }
    }
    if (j < n) partial[(size_t)blockIdx.y * n + j] = make_double2(ar, ai);
}

// Tabulated form: H0(k sqrt(t)) from the per-operator octave table (lsgpu::H0Table)
// held in shared memory: coef [ncell][NC] double2, then (mid, inv_hw) [ncell],
// then (base, shift) [noct].  Pairs with t outside the table use ls_h0_r2.
// NC = polynomial degree + 1; the autotuner of the operator setup picks NC.
template <int NC_TAB>
__global__ void __launch_bounds__(PS_TPB) k_pairsum_tab(const double2* __restrict__ xy, const double* __restrict__ w,
                                                        const double2* __restrict__ m, const double2* __restrict__ f,
                                                        int n, int src_per_chunk, double k, double inv_k,
                                                        const double2* __restrict__ tab_g, int ncell, int noct, int b_lo,
                                                        double2* __restrict__ partial) {
    extern __shared__ double2 tab[];
    __shared__ double4 tile[PS_TILE];
    const int words = ncell * (NC_TAB + 1) + (noct + 1) / 2;      // double2 words
    for (int i = threadIdx.x; i < words; i += PS_TPB) tab[i] = tab_g[i];
    const double2* coef = tab;
    const double2* mh = tab + (size_t)ncell * NC_TAB;
    const int2* oct = reinterpret_cast<const int2*>(mh + ncell);
    const int j = blockIdx.x * PS_TPB + threadIdx.x;
    const int s_begin = blockIdx.y * src_per_chunk;
    const int s_end = min(n, s_begin + src_per_chunk);
    const double2 yj = xy[min(j, n - 1)];
    double ar = 0.0, ai = 0.0;
    for (int base = s_begin; base < s_end; base += PS_TILE) {
        __syncthreads();
        for (int i = threadIdx.x; i < PS_TILE; i += PS_TPB) {
            int src = base + i;
            double4 v = make_double4(0.0, 0.0, 0.0, 0.0);
            if (src < s_end) {
                double2 p = xy[src];
                double2 ff = f[src];
                if (m) ff = cmul(m[src], ff);
                double ww = w ? w[src] : 1.0;
                v = make_double4(p.x, p.y, ww * ff.x, ww * ff.y);
            }
            tile[i] = v;
        }
        __syncthreads();
        const int cnt = min(PS_TILE, s_end - base);
        for (int i = 0; i < cnt; ++i) {
            double4 s = tile[i];
            double dx = yj.x - s.x, dy = yj.y - s.y;
            double t = fma(dx, dx, dy * dy);
            int hi = __double2hiint(t);
            unsigned o = (unsigned)((hi >> 20) - b_lo);
            double hr, him;
            if (o < (unsigned)noct) {
                int2 ob = oct[o];
                int cell = ob.x + ((hi & 0xfffff) >> ob.y);
                double2 q = mh[cell];
                double u = (t - q.x) * q.y;
                const double2* c = coef + (size_t)cell * NC_TAB;
                double2 cc = c[NC_TAB - 1];
                hr = cc.x;
                him = cc.y;
#pragma unroll
                for (int e = NC_TAB - 2; e >= 0; --e) {
                    cc = c[e];
                    hr = fma(hr, u, cc.x);
                    him = fma(him, u, cc.y);
                }
            } else if (t > 0.0) {
                double2 h = ls_h0_r2(t, k, inv_k);
                hr = h.x;
                him = h.y;
            } else {
                continue;                     // the self pair
            }
            ar = fma(hr, s.z, fma(-him, s.w, ar));
            ai = fma(hr, s.w, fma(him, s.z, ai));
        }
    }
    if (j < n) partial[(size_t)blockIdx.y * n + j] = make_double2(ar, ai);
}

// Precision form: FP32 pair sum.  Coordinates travel as float pairs (hi, lo);
// dx, dy and t = dx^2 + dy^2 are formed in double-float arithmetic (TwoSum /
// FMA-based TwoProduct) so that t keeps a relative error near 1e-14 and the
// cell variable u near 1e-7; H0 comes from an FP32 table (complex64 degree-6
// polynomials, validated to 2e-8 at setup); terms are accumulated with Kahan
// compensation in FP32.  Pairs below the table range use the FP64 routine.
#define NC_F32 7
struct F32Tile { float4 xy; float2 s; };

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bv = s - a;
    float av = s - bv;
    e = (a - av) + (b - bv);
}

__device__ __forceinline__ void df_diff(float ah, float al, float bh, float bl, float& dh, float& dl) {
    float s, e;
    two_sum(ah, -bh, s, e);
    e += al - bl;
    dh = s + e;
    dl = e - (dh - s);
}

// H0(k |y - x|) from the FP32 table for target (txh + txl, tyh + tyl) and source coordinates
// sxy = (x_h, x_l, y_h, y_l): double-float differences and t, FP32 cell variable and Horner,
// the FP64 routine outside the table range.  Returns false (H = 0) for t = 0, the self pair.
__device__ __forceinline__ bool f32_h0(float txh, float txl, float tyh, float tyl, float4 sxy, const float2* coef,
                                       const float4* cellv, const int2* oct, int noct, int b_lo, double k, double inv_k,
                                       float& hr, float& him) {
    float dxh, dxl, dyh, dyl;
    df_diff(txh, txl, sxy.x, sxy.y, dxh, dxl);
    df_diff(tyh, tyl, sxy.z, sxy.w, dyh, dyl);
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
    int bits = __float_as_int(th);
    unsigned o = (unsigned)((bits >> 23) - b_lo);
    if (o < (unsigned)noct) {
        int2 ob = oct[o];
        int cell = ob.x + ((bits & 0x7fffff) >> ob.y);
        float4 cv = cellv[cell];
        float u = ((th - cv.x) + (tl - cv.y)) * cv.z;
        const float2* c = coef + cell * NC_F32;
        float2 cc = c[NC_F32 - 1];
        hr = cc.x;
        him = cc.y;
#pragma unroll
        for (int e = NC_F32 - 2; e >= 0; --e) {
            cc = c[e];
            hr = fmaf(hr, u, cc.x);
            him = fmaf(him, u, cc.y);
        }
        return true;
    }
    if (th > 0.f) {
        double2 h = ls_h0_r2((double)th + (double)tl, k, inv_k);
        hr = (float)h.x;
        him = (float)h.y;
        return true;
    }
    hr = 0.f;
    him = 0.f;
    return false;
}

__global__ void __launch_bounds__(PS_TPB) k_pairsum_f32(const double2* __restrict__ xy, const double* __restrict__ w,
                                                        const double2* __restrict__ m, const double2* __restrict__ f,
                                                        int n, int src_per_chunk, double k, double inv_k,
                                                        const float4* __restrict__ tab_g, int ncell, int noct, int b_lo,
                                                        double2* __restrict__ partial) {
    extern __shared__ float4 ftab[];
    __shared__ F32Tile tile[PS_TILE];
    // layout: coef [ncell][NC_F32] float2 (as float4 pairs), cell (mid_hi, mid_lo, inv_hw, 0) [ncell], oct int2 [noct]
    const int coef_f4 = (ncell * NC_F32 + 1) / 2;
    const int words = coef_f4 + ncell + (noct + 1) / 2;
    for (int i = threadIdx.x; i < words; i += PS_TPB) ftab[i] = tab_g[i];
    const float2* coef = reinterpret_cast<const float2*>(ftab);
    const float4* cellv = ftab + coef_f4;
    const int2* oct = reinterpret_cast<const int2*>(cellv + ncell);
    const int j = blockIdx.x * PS_TPB + threadIdx.x;
    const int s_begin = blockIdx.y * src_per_chunk;
    const int s_end = min(n, s_begin + src_per_chunk);
    const double2 yj = xy[min(j, n - 1)];
    const float txh = (float)yj.x, txl = (float)(yj.x - (double)txh);
    const float tyh = (float)yj.y, tyl = (float)(yj.y - (double)tyh);
    float sr = 0.f, si = 0.f, cr = 0.f, ci = 0.f;     // Kahan sums and compensations
    for (int base = s_begin; base < s_end; base += PS_TILE) {
        __syncthreads();
        for (int i = threadIdx.x; i < PS_TILE; i += PS_TPB) {
            int src = base + i;
            F32Tile v;
            v.xy = make_float4(0.f, 0.f, 0.f, 0.f);
            v.s = make_float2(0.f, 0.f);
            if (src < s_end) {
                double2 p = xy[src];
                double2 ff = f[src];
                if (m) ff = cmul(m[src], ff);
                double ww = w ? w[src] : 1.0;
                float xh = (float)p.x, yh = (float)p.y;
                v.xy = make_float4(xh, (float)(p.x - (double)xh), yh, (float)(p.y - (double)yh));
                v.s = make_float2((float)(ww * ff.x), (float)(ww * ff.y));
            }
            tile[i] = v;
        }
        __syncthreads();
        const int cnt = min(PS_TILE, s_end - base);
        for (int i = 0; i < cnt; ++i) {
            F32Tile src = tile[i];
            float hr, him;
            if (!f32_h0(txh, txl, tyh, tyl, src.xy, coef, cellv, oct, noct, b_lo, k, inv_k, hr, him))
                continue;                     // the self pair
            float tr = fmaf(hr, src.s.x, -him * src.s.y);
            float ti = fmaf(hr, src.s.y, him * src.s.x);
            float yr = tr - cr, yi = ti - ci;
            float nr = sr + yr, ni = si + yi;
            cr = (nr - sr) - yr;
            ci = (ni - si) - yi;
            sr = nr;
            si = ni;
        }
    }
    if (j < n) partial[(size_t)blockIdx.y * n + j] = make_double2((double)sr - (double)cr, (double)si - (double)ci);
}

// Kahan step: (s, c) += v
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// The precision form's pair sum over unordered pairs: the decomposition and lane rotation
// of k_pairsum_dfs (strips of 128 targets, circular block distances split in chunks,
// chunk 0 also the diagonal block; rows to partial[c], columns to partial[nchunk + d - 1])
// with the arithmetic of k_pairsum_f32 (FP32 table, double-float t, Kahan-compensated FP32
// sums, folded into FP64 once per 128-source unit).
__global__ void __launch_bounds__(PS_TPB) k_pairsum_f32s(const double2* __restrict__ xy, const double* __restrict__ w,
                                                         const double2* __restrict__ m, const double2* __restrict__ f,
                                                         int n, int nb, int dper, double k, double inv_k,
                                                         const float4* __restrict__ tab_g, int ncell, int noct, int b_lo,
                                                         double2* __restrict__ partial) {
    extern __shared__ float4 ftab[];
    __shared__ F32Tile tile[PS_TPB];
    __shared__ float2 colbuf[PS_TPB / 32][PS_TPB];
    const int coef_f4 = (ncell * NC_F32 + 1) / 2;
    const int words = coef_f4 + ncell + (noct + 1) / 2;
    for (int i = threadIdx.x; i < words; i += PS_TPB) ftab[i] = tab_g[i];
    const float2* coef = reinterpret_cast<const float2*>(ftab);
    const float4* cellv = ftab + coef_f4;
    const int2* oct = reinterpret_cast<const int2*>(cellv + ncell);
    const int I = blockIdx.x, c = blockIdx.y, nchunk = gridDim.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = I * PS_TPB + threadIdx.x;
    const int D = nb / 2;
    auto load_tile = [&](int blk) {
        const int q = blk * PS_TPB + threadIdx.x;
        F32Tile v;
        v.xy = make_float4(0.f, 0.f, 0.f, 0.f);
        v.s = make_float2(0.f, 0.f);
        if (q < n) {
            double2 p = xy[q];
            double2 ff = f[q];
            if (m) ff = cmul(m[q], ff);
            double ww = w ? w[q] : 1.0;
            float xh = (float)p.x, yh = (float)p.y;
            v.xy = make_float4(xh, (float)(p.x - (double)xh), yh, (float)(p.y - (double)yh));
            v.s = make_float2((float)(ww * ff.x), (float)(ww * ff.y));
        }
        tile[threadIdx.x] = v;
    };
    __syncthreads();
    load_tile(I);
    __syncthreads();
    const float2 s_me = tile[threadIdx.x].s;
    const double2 yi = xy[min(i, n - 1)];
    const float txh = (float)yi.x, txl = (float)(yi.x - (double)txh);
    const float tyh = (float)yi.y, tyl = (float)(yi.y - (double)tyh);
    double accr = 0.0, acci = 0.0;
    if (c == 0) {                          // the diagonal block: ordered pairs, rows only
        float sr = 0.f, si = 0.f, er = 0.f, ei = 0.f;
        for (int q = 0; q < PS_TPB; ++q) {
            if (q == (int)threadIdx.x) continue;
            const F32Tile src = tile[q];
            float hr, him;
            if (!f32_h0(txh, txl, tyh, tyl, src.xy, coef, cellv, oct, noct, b_lo, k, inv_k, hr, him)) continue;
            kahan_add(sr, er, fmaf(hr, src.s.x, -him * src.s.y));
            kahan_add(si, ei, fmaf(hr, src.s.y, him * src.s.x));
        }
        accr += (double)sr - (double)er;
        acci += (double)si - (double)ei;
    }
    const int d0 = 1 + c * dper, d1 = min(D, (c + 1) * dper);
    for (int d = d0; d <= d1; ++d) {
        if (2 * D == nb && d == D && I >= D) continue;      // that block pair belongs to strip I - D
        const int J = (I + d) % nb;
        __syncthreads();
        load_tile(J);
        __syncthreads();
        float sr = 0.f, si = 0.f, er = 0.f, ei = 0.f;
#pragma unroll 1
        for (int sub = 0; sub < PS_TPB / 32; ++sub) {
            float cr = 0.f, ci = 0.f, ecr = 0.f, eci = 0.f;
#pragma unroll 2
            for (int r = 0; r < 32; ++r) {
                const F32Tile src = tile[sub * 32 + ((lane + r) & 31)];
                float hr, him;
                f32_h0(txh, txl, tyh, tyl, src.xy, coef, cellv, oct, noct, b_lo, k, inv_k, hr, him);
                kahan_add(sr, er, fmaf(hr, src.s.x, -him * src.s.y));
                kahan_add(si, ei, fmaf(hr, src.s.y, him * src.s.x));
                kahan_add(cr, ecr, fmaf(hr, s_me.x, -him * s_me.y));
                kahan_add(ci, eci, fmaf(hr, s_me.y, him * s_me.x));
                const int from = (lane + 1) & 31;
                cr = __shfl_sync(0xffffffffu, cr, from);
                ci = __shfl_sync(0xffffffffu, ci, from);
                ecr = __shfl_sync(0xffffffffu, ecr, from);
                eci = __shfl_sync(0xffffffffu, eci, from);
            }
            colbuf[warp][sub * 32 + lane] = make_float2(cr - ecr, ci - eci);
        }
        accr += (double)sr - (double)er;
        acci += (double)si - (double)ei;
        __syncthreads();
        const int jj = J * PS_TPB + threadIdx.x;
        if (jj < n) {
            double tr = 0.0, ti = 0.0;
#pragma unroll
            for (int wv = 0; wv < PS_TPB / 32; ++wv) {
                tr += (double)colbuf[wv][threadIdx.x].x;
                ti += (double)colbuf[wv][threadIdx.x].y;
            }
            partial[(size_t)(nchunk + d - 1) * n + jj] = make_double2(tr, ti);
        }
    }
    if (i < n) partial[(size_t)c * n + i] = make_double2(accr, acci);
}

// FP64-accurate pair sum in double-float (pairs of FP32, ~48-bit significand) on the
// FP32 pipe (pairsum = 3): DF coordinate differences, DF t = dx^2 + dy^2, exact DF
// cell variable u (t and the cell centre share an octave, so t_hi - mid_hi is exact,
// and 1/half-width is a power of two), DF Horner on the degree-11 table stored as
// (hi, lo) float pairs, DF complex multiply-accumulate per 256-source tile folded
// into FP64.  Error-free transformations: TwoSum (Knuth), TwoProduct via FMA.
struct DF { float h, l; };
__device__ __forceinline__ DF df_fast(float a, float b) {       // |a| >= |b|
    float s = a + b;
    return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    e += a.l + b.l;
    return df_fast(s, e);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return df_fast(p, e);
}
// a * u + c
__device__ __forceinline__ DF df_mad(DF a, DF u, DF c) {
    float p = a.h * u.h;
    float e = fmaf(a.h, u.h, -p);
    float s, e2;
    two_sum(p, c.h, s, e2);
    e = fmaf(a.h, u.l, e);
    e = fmaf(a.l, u.h, e);
    e += e2 + c.l;
    return df_fast(s, e);
}
__device__ __forceinline__ DF df_from(double x) {
    float h = (float)x;
    return DF{h, (float)(x - (double)h)};
}

struct DFTile { float4 xy; float4 s; };     // (x_h, x_l, y_h, y_l), (s_re_h, s_re_l, s_im_h, s_im_l)

// H0(k |y - x|) in double-float for target (tx, ty) and source coordinates sxy = (x_h, x_l,
// y_h, y_l): DF coordinate differences, DF t = dx^2 + dy^2, exact DF cell variable u (t and
// the cell centre share an octave, so t_hi - mid_hi is exact, and 1/half-width is a power of
// two), DF Horner on the table (the top NF steps in plain FP32), the FP64 routine outside the
// table range.  Returns false (H = 0) for t = 0, the self pair.
template <int NC_TAB, int NF>
__device__ __forceinline__ bool df_h0(DF tx, DF ty, float4 sxy, const float4* coef, const float4* cellv,
                                      const int2* oct, int noct, int b_lo, double k, double inv_k, DF& hr, DF& hi) {
    float dxh, dxl, dyh, dyl;
    df_diff(tx.h, tx.l, sxy.x, sxy.y, dxh, dxl);
    df_diff(ty.h, ty.l, sxy.z, sxy.w, dyh, dyl);
    float p1 = dxh * dxh, e1 = fmaf(dxh, dxh, -p1);
    e1 = fmaf(2.f * dxh, dxl, e1);
    float p2 = dyh * dyh, e2 = fmaf(dyh, dyh, -p2);
    e2 = fmaf(2.f * dyh, dyl, e2);
    float th, tl;
    two_sum(p1, p2, th, tl);
    tl += e1 + e2;
    DF t = df_fast(th, tl);
    int bits = __float_as_int(t.h);
    unsigned o = (unsigned)((bits >> 23) - b_lo);
    if (o < (unsigned)noct) {
        int2 ob = oct[o];
        int cell = ob.x + ((bits & 0x7fffff) >> ob.y);
        float4 cv = cellv[cell];
        float d0, d1;
        two_sum(t.h - cv.x, t.l - cv.y, d0, d1);      // t.h - mid.h is exact
        DF u = DF{d0 * cv.z, d1 * cv.z};                // times a power of two: exact
        const float4* c = coef + (size_t)cell * NC_TAB;
        float4 cc = c[NC_TAB - 1];
        // compensated Horner: the FP32 Horner value (sr, si) and its running correction
        // (kr, ki); each step adds the TwoProd residual of s u_h, the TwoSum residual of
        // s u_h + a_h, the low parts a_l and s u_l, and the correction times u_h
        float sr = cc.x, si = cc.z, kr = 0.f, ki = 0.f;
        if (NF > 0) {
#pragma unroll
            for (int e = NC_TAB - 2; e >= NC_TAB - NF; --e) {
                cc = c[e];
                sr = fmaf(sr, u.h, cc.x);
                si = fmaf(si, u.h, cc.z);
            }
        } else {
            kr = cc.y;
            ki = cc.w;
        }
#pragma unroll
        for (int e = (NF > 0 ? NC_TAB - NF : NC_TAB - 1) - 1; e >= 0; --e) {
            cc = c[e];
            const float pr = sr * u.h, pi_r = fmaf(sr, u.h, -pr);
            const float pm = si * u.h, pi_m = fmaf(si, u.h, -pm);
            float tr, er, tm, em;
            two_sum(pr, cc.x, tr, er);
            two_sum(pm, cc.z, tm, em);
            kr = fmaf(kr, u.h, fmaf(sr, u.l, (pi_r + er) + cc.y));
            ki = fmaf(ki, u.h, fmaf(si, u.l, (pi_m + em) + cc.w));
            sr = tr;
            si = tm;
        }
        hr = df_fast(sr, kr);
        hi = df_fast(si, ki);
        return true;
    }
    if (t.h > 0.f) {
        double2 h = ls_h0_r2((double)t.h + (double)t.l, k, inv_k);
        hr = df_from(h.x);
        hi = df_from(h.y);
        return true;
    }
    hr = DF{0.f, 0.f};
    hi = DF{0.f, 0.f};
    return false;
}

// acc += h * s (complex, double-float)
__device__ __forceinline__ void df_cmac(DF hr, DF hi, DF s_re, DF s_im, DF& ar, DF& ai) {
    DF a1 = df_mul(hr, s_re), a2 = df_mul(hi, s_im), a3 = df_mul(hr, s_im), a4 = df_mul(hi, s_re);
    ar = df_add(ar, df_add(a1, DF{-a2.h, -a2.l}));
    ai = df_add(ai, df_add(a3, a4));
}

// The same with an unnormalised accumulator (ar.h, ar.l), (ai.h, ai.l): each product is
// formed to first order (high product, its FMA residual, the two cross terms), the high
// parts are added with TwoSum and every residual goes into the low word; normalise with
// df_fast before the low word can grow past 2^-24 of the high one (here: every 32 to 128
// terms, whose residuals are each below 2^-23 of their product).
__device__ __forceinline__ void df_cmac_lazy(DF hr, DF hi, float4 sv, DF& ar, DF& ai) {
    const float p1 = hr.h * sv.x, p2 = hi.h * sv.z, p3 = hr.h * sv.z, p4 = hi.h * sv.x;
    float e1 = fmaf(hr.h, sv.x, -p1), e2 = fmaf(hi.h, sv.z, -p2);
    float e3 = fmaf(hr.h, sv.z, -p3), e4 = fmaf(hi.h, sv.x, -p4);
    e1 = fmaf(hr.l, sv.x, fmaf(hr.h, sv.y, e1));
    e2 = fmaf(hi.l, sv.z, fmaf(hi.h, sv.w, e2));
    e3 = fmaf(hr.l, sv.z, fmaf(hr.h, sv.w, e3));
    e4 = fmaf(hi.l, sv.x, fmaf(hi.h, sv.y, e4));
    float t, err;
    two_sum(ar.h, p1, t, err);
    ar.l += err + e1;
    two_sum(t, -p2, ar.h, err);
    ar.l += err - e2;
    two_sum(ai.h, p3, t, err);
    ai.l += err + e3;
    two_sum(t, p4, ai.h, err);
    ai.l += err + e4;
}

// NF > 0: the top NF coefficients of the Horner chain (whose terms are below 2^-24 of |H0|
// on every cell, checked when the table is uploaded) are summed in plain FP32, the rest in
// double-float.
template <int NC_TAB, int NF>
__global__ void __launch_bounds__(PS_TPB) k_pairsum_df(const double2* __restrict__ xy, const double* __restrict__ w,
                                                       const double2* __restrict__ m, const double2* __restrict__ f,
                                                       int n, int src_per_chunk, double k, double inv_k,
                                                       const float4* __restrict__ tab_g, int ncell, int noct, int b_lo,
                                                       double2* __restrict__ partial) {
    // table layout (float4 words): coef [ncell][NC_TAB] as (re_h, re_l, im_h, im_l),
    // cells (mid_h, mid_l, inv_hw, 0) [ncell], oct int2 (base, 23 - m) [noct]
    extern __shared__ float4 dtab[];
    __shared__ DFTile tile[PS_TILE];
    const int words = ncell * (NC_TAB + 1) + (noct + 1) / 2;
    for (int i = threadIdx.x; i < words; i += PS_TPB) dtab[i] = tab_g[i];
    const float4* coef = dtab;
    const float4* cellv = dtab + (size_t)ncell * NC_TAB;
    const int2* oct = reinterpret_cast<const int2*>(cellv + ncell);
    const int j = blockIdx.x * PS_TPB + threadIdx.x;
    const int s_begin = blockIdx.y * src_per_chunk;
    const int s_end = min(n, s_begin + src_per_chunk);
    const double2 yj = xy[min(j, n - 1)];
    const DF tx = df_from(yj.x), ty = df_from(yj.y);
    double accr = 0.0, acci = 0.0;
    for (int base = s_begin; base < s_end; base += PS_TILE) {
        __syncthreads();
        for (int i = threadIdx.x; i < PS_TILE; i += PS_TPB) {
            int src = base + i;
            DFTile v;
            v.xy = make_float4(0.f, 0.f, 0.f, 0.f);
            v.s = make_float4(0.f, 0.f, 0.f, 0.f);
            if (src < s_end) {
                double2 p = xy[src];
                double2 ff = f[src];
                if (m) ff = cmul(m[src], ff);
                double ww = w ? w[src] : 1.0;
                DF a = df_from(p.x), b = df_from(p.y), c = df_from(ww * ff.x), d = df_from(ww * ff.y);
                v.xy = make_float4(a.h, a.l, b.h, b.l);
                v.s = make_float4(c.h, c.l, d.h, d.l);
            }
            tile[i] = v;
        }
        __syncthreads();
        DF sr{0.f, 0.f}, si{0.f, 0.f};
        const int cnt = min(PS_TILE, s_end - base);
        for (int i = 0; i < cnt; ++i) {
            DFTile src = tile[i];
            DF hr, hi;
            if (!df_h0<NC_TAB, NF>(tx, ty, src.xy, coef, cellv, oct, noct, b_lo, k, inv_k, hr, hi))
                continue;                     // the self pair
            DF s_re{src.s.x, src.s.y}, s_im{src.s.z, src.s.w};
            DF a1 = df_mul(hr, s_re), a2 = df_mul(hi, s_im), a3 = df_mul(hr, s_im), a4 = df_mul(hi, s_re);
            sr = df_add(sr, df_add(a1, DF{-a2.h, -a2.l}));
            si = df_add(si, df_add(a3, a4));
        }
        accr += (double)sr.h + (double)sr.l;
        acci += (double)si.h + (double)si.l;
    }
    if (j < n) partial[(size_t)blockIdx.y * n + j] = make_double2(accr, acci);
}

// The same pair sum using the symmetry H(i, j) = H(j, i): every unordered pair is evaluated
// once and feeds both the row sum of its target and the column sum of its source.
// The nodes form nb blocks of 128 placed on a circle; strip I (blockIdx.x) pairs with the
// blocks at circular distance d = 1 .. D after it, D = floor(nb / 2) (the distance nb / 2 of
// an even nb only from I < nb / 2, so each unordered block pair occurs once), the distances
// split into gridDim.y chunks of dper, one CTA per (strip, chunk); chunk 0 also takes the
// diagonal block (ordered pairs i != j, rows only).  Deterministic output, no atomics:
//   row sums     partial[c][I*128 + t]              c = chunk
//   column sums  partial[nchunk + d - 1][J*128 + t]  J = (I + d) mod nb
// (for an even nb the slot of d = nb / 2 of the blocks J < nb / 2 is left to the caller to
// zero).  In a unit (I, J) a warp owns 32 targets and walks each 32-source sub-block of J
// in 32 steps: at step r lane l pairs its target with source (l + r) mod 32 and carries
// that source's column accumulator, passed to lane l - 1 after the step, so that after the
// 32 steps lane l holds the sum for source l over the warp's targets; the four warps'
// sums are added in shared memory.  Arithmetic per pair as k_pairsum_df.
template <int NC_TAB, int NF>
__global__ void __launch_bounds__(PS_TPB) k_pairsum_dfs(const double2* __restrict__ xy, const double* __restrict__ w,
                                                        const double2* __restrict__ m, const double2* __restrict__ f,
                                                        int n, int nb, int dper, double k, double inv_k,
                                                        const float4* __restrict__ tab_g, int ncell, int noct, int b_lo,
                                                        double2* __restrict__ partial) {
    extern __shared__ float4 dtab[];
    __shared__ DFTile tile[PS_TPB];
    __shared__ float4 colbuf[PS_TPB / 32][PS_TPB];
    const int words = ncell * (NC_TAB + 1) + (noct + 1) / 2;
    for (int i = threadIdx.x; i < words; i += PS_TPB) dtab[i] = tab_g[i];
    const float4* coef = dtab;
    const float4* cellv = dtab + (size_t)ncell * NC_TAB;
    const int2* oct = reinterpret_cast<const int2*>(cellv + ncell);
    const int I = blockIdx.x, c = blockIdx.y, nchunk = gridDim.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = I * PS_TPB + threadIdx.x;
    const int D = nb / 2;
    // the strength of node q, (w m f)_q, as a DF tile entry (zero past n)
    auto load_tile = [&](int blk) {
        const int q = blk * PS_TPB + threadIdx.x;
        DFTile v;
        v.xy = make_float4(0.f, 0.f, 0.f, 0.f);
        v.s = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < n) {
            double2 p = xy[q];
            double2 ff = f[q];
            if (m) ff = cmul(m[q], ff);
            double ww = w ? w[q] : 1.0;
            DF a = df_from(p.x), b = df_from(p.y), cr = df_from(ww * ff.x), ci = df_from(ww * ff.y);
            v.xy = make_float4(a.h, a.l, b.h, b.l);
            v.s = make_float4(cr.h, cr.l, ci.h, ci.l);
        }
        tile[threadIdx.x] = v;
    };
    // this thread's target and its own strength (for the column sums)
    __syncthreads();
    load_tile(I);
    __syncthreads();
    const DFTile me = tile[threadIdx.x];
    const double2 yi = xy[min(i, n - 1)];
    const DF tx = df_from(yi.x), ty = df_from(yi.y);
    double accr = 0.0, acci = 0.0;
    if (c == 0) {                          // the diagonal block: ordered pairs, rows only
        DF sr{0.f, 0.f}, sim{0.f, 0.f};
        for (int q = 0; q < PS_TPB; ++q) {
            const DFTile src = tile[q];
            DF hr, hi;
            if (q != (int)threadIdx.x &&
                df_h0<NC_TAB, NF>(tx, ty, src.xy, coef, cellv, oct, noct, b_lo, k, inv_k, hr, hi))
                df_cmac_lazy(hr, hi, src.s, sr, sim);
            if ((q & 31) == 31) {
                sr = df_fast(sr.h, sr.l);
                sim = df_fast(sim.h, sim.l);
            }
        }
        accr += (double)sr.h + (double)sr.l;
        acci += (double)sim.h + (double)sim.l;
    }
    const int d0 = 1 + c * dper, d1 = min(D, (c + 1) * dper);
    for (int d = d0; d <= d1; ++d) {
        if (2 * D == nb && d == D && I >= D) continue;      // that block pair belongs to strip I - D
        const int J = (I + d) % nb;
        __syncthreads();
        load_tile(J);
        __syncthreads();
        DF sr{0.f, 0.f}, sim{0.f, 0.f};
#pragma unroll 1
        for (int sub = 0; sub < PS_TPB / 32; ++sub) {
            DF cr{0.f, 0.f}, ci{0.f, 0.f};
#pragma unroll 2
            for (int r = 0; r < 32; ++r) {
                const DFTile src = tile[sub * 32 + ((lane + r) & 31)];
                DF hr, hi;
                df_h0<NC_TAB, NF>(tx, ty, src.xy, coef, cellv, oct, noct, b_lo, k, inv_k, hr, hi);
                df_cmac_lazy(hr, hi, src.s, sr, sim);
                df_cmac_lazy(hr, hi, me.s, cr, ci);
                const int from = (lane + 1) & 31;
                cr.h = __shfl_sync(0xffffffffu, cr.h, from);
                cr.l = __shfl_sync(0xffffffffu, cr.l, from);
                ci.h = __shfl_sync(0xffffffffu, ci.h, from);
                ci.l = __shfl_sync(0xffffffffu, ci.l, from);
            }
            cr = df_fast(cr.h, cr.l);
            ci = df_fast(ci.h, ci.l);
            colbuf[warp][sub * 32 + lane] = make_float4(cr.h, cr.l, ci.h, ci.l);
            sr = df_fast(sr.h, sr.l);             // keep the row's low word small (32 terms per step)
            sim = df_fast(sim.h, sim.l);
        }
        accr += (double)sr.h + (double)sr.l;
        acci += (double)sim.h + (double)sim.l;
        __syncthreads();
        const int jj = J * PS_TPB + threadIdx.x;
        if (jj < n) {
            DF tr{0.f, 0.f}, ti{0.f, 0.f};
#pragma unroll
            for (int wv = 0; wv < PS_TPB / 32; ++wv) {
                const float4 v = colbuf[wv][threadIdx.x];
                tr = df_add(tr, DF{v.x, v.y});
                ti = df_add(ti, DF{v.z, v.w});
            }
            partial[(size_t)(nchunk + d - 1) * n + jj] = make_double2((double)tr.h + (double)tr.l,
                                                                      (double)ti.h + (double)ti.l);
        }
    }
    if (i < n) partial[(size_t)c * n + i] = make_double2(accr, acci);
}

// Batched form: R right-hand sides.  Each thread owns one target and a block of
// RB right-hand sides; H(j, n) is generated once per pair from the FP32 table
// (double-float t as in k_pairsum_f32) and applied to the RB strengths.  Sums
// are Kahan-compensated FP32 over runs of 64 sources, folded into FP64
// accumulators after each run.
//   f [R][n] densities; partial [R][nchunk][n] (blockIdx.z = RHS block).
#define MRB 8

// One work unit of the batched pair sum: target block tb, source chunk, RHS block rb.
struct MultiArgs {
    const double2* xy;
    const double* w;
    const double2* m;
    const double2* f;
    size_t sf;
    int n, R, spc, nchunk;
    double k, inv_k;
    int ncell, noct, b_lo;
    double2* partial;
};

__device__ __forceinline__ void multi_unit(const MultiArgs& A, int tb, int chunk, int rb, const float4* ftab,
                                           float4* txy, float2 (*ts)[MRB]) {
    const int coef_f4 = (A.ncell * NC_F32 + 1) / 2;
    const float2* coef = reinterpret_cast<const float2*>(ftab);
    const float4* cellv = ftab + coef_f4;
    const int2* oct = reinterpret_cast<const int2*>(cellv + A.ncell);
    const int n = A.n;
    const int j = tb * PS_TPB + threadIdx.x;
    const int r0 = rb * MRB;
    const int nr = min(MRB, A.R - r0);
    const int s_begin = chunk * A.spc;
    const int s_end = min(n, s_begin + A.spc);
    const double2 yj = A.xy[min(j, n - 1)];
    const float txh = (float)yj.x, txl = (float)(yj.x - (double)txh);
    const float tyh = (float)yj.y, tyl = (float)(yj.y - (double)tyh);
    double accr[MRB], acci[MRB];
#pragma unroll
    for (int q = 0; q < MRB; ++q) { accr[q] = 0.0; acci[q] = 0.0; }
    for (int base = s_begin; base < s_end; base += PS_TILE) {
        __syncthreads();
        for (int i = threadIdx.x; i < PS_TILE; i += PS_TPB) {
            int src = base + i;
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
            if (src < s_end) {
                double2 p = A.xy[src];
                float xh = (float)p.x, yh = (float)p.y;
                c = make_float4(xh, (float)(p.x - (double)xh), yh, (float)(p.y - (double)yh));
            }
            txy[i] = c;
            double ww = (src < s_end) ? (A.w ? A.w[src] : 1.0) : 0.0;
            double2 mm = (src < s_end && A.m) ? A.m[src] : make_double2(1.0, 0.0);
#pragma unroll
            for (int q = 0; q < MRB; ++q) {
                float2 v = make_float2(0.f, 0.f);
                if (src < s_end && q < nr) {
                    double2 ff = cmul(mm, A.f[(size_t)(r0 + q) * A.sf + src]);
                    v = make_float2((float)(ww * ff.x), (float)(ww * ff.y));
                }
                ts[i][q] = v;
            }
        }
        __syncthreads();
        const int cnt = min(PS_TILE, s_end - base);
        // Kahan-compensated FP32 sums over runs of 64 sources, folded into the FP64
        // accumulators after each run
        for (int i0 = 0; i0 < cnt; i0 += 64) {
            float sr[MRB], si[MRB], cr[MRB], ci[MRB];
#pragma unroll
            for (int q = 0; q < MRB; ++q) { sr[q] = 0.f; si[q] = 0.f; cr[q] = 0.f; ci[q] = 0.f; }
            const int i1 = min(cnt, i0 + 64);
            for (int i = i0; i < i1; ++i) {
                float4 sc = txy[i];
                float dxh, dxl, dyh, dyl;
                df_diff(txh, txl, sc.x, sc.y, dxh, dxl);
                df_diff(tyh, tyl, sc.z, sc.w, dyh, dyl);
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
                int bits = __float_as_int(th);
                unsigned o = (unsigned)((bits >> 23) - A.b_lo);
                float hr, him;
                if (o < (unsigned)A.noct) {
                    int2 ob = oct[o];
                    int cell = ob.x + ((bits & 0x7fffff) >> ob.y);
                    float4 cv = cellv[cell];
                    float u = ((th - cv.x) + (tl - cv.y)) * cv.z;
                    const float2* c = coef + cell * NC_F32;
                    float2 cc = c[NC_F32 - 1];
                    hr = cc.x;
                    him = cc.y;
#pragma unroll
                    for (int e = NC_F32 - 2; e >= 0; --e) {
                        cc = c[e];
                        hr = fmaf(hr, u, cc.x);
                        him = fmaf(him, u, cc.y);
                    }
                } else if (th > 0.f) {
                    double2 h = ls_h0_r2((double)th + (double)tl, A.k, A.inv_k);
                    hr = (float)h.x;
                    him = (float)h.y;
                } else {
                    continue;
                }
#pragma unroll
                for (int q = 0; q < MRB; ++q) {
                    float2 v = ts[i][q];
                    float tr = fmaf(hr, v.x, -him * v.y) - cr[q];
                    float ti = fmaf(hr, v.y, him * v.x) - ci[q];
                    float nr = sr[q] + tr, ni = si[q] + ti;
                    cr[q] = (nr - sr[q]) - tr;
                    ci[q] = (ni - si[q]) - ti;
                    sr[q] = nr;
                    si[q] = ni;
                }
            }
#pragma unroll
            for (int q = 0; q < MRB; ++q) {
                accr[q] += (double)sr[q] - (double)cr[q];
                acci[q] += (double)si[q] - (double)ci[q];
            }
        }
    }
    if (j < n)
        for (int q = 0; q < nr; ++q)
            A.partial[((size_t)(r0 + q) * A.nchunk + chunk) * n + j] = make_double2(accr[q], acci[q]);
}

__global__ void __launch_bounds__(PS_TPB) k_pairsum_multi_f32(MultiArgs A, const float4* __restrict__ tab_g) {
    extern __shared__ float4 ftab[];
    __shared__ float4 txy[PS_TILE];
    __shared__ float2 ts[PS_TILE][MRB];
    const int words = (A.ncell * NC_F32 + 1) / 2 + A.ncell + (A.noct + 1) / 2;
    for (int i = threadIdx.x; i < words; i += PS_TPB) ftab[i] = tab_g[i];
    multi_unit(A, blockIdx.x, blockIdx.y, blockIdx.z, ftab, txy, ts);
}

// The batched pair sum in double-float (FP64-accurate), for the residuals of the batched
// solves' refinement: the decomposition of k_pairsum_multi_f32 (target block x source chunk
// x block of MRB right-hand sides), H from the double-float table (df_h0), the densities as
// double-float pairs, and per right-hand side an accumulator kept as (hi, lo): each product
// H s is formed exactly to first order (hi product, its FMA residual and the cross terms),
// the hi parts added with TwoSum, the residuals into lo; folded into FP64 every
// MDF_TILE sources.
#define MDF_TILE 64
template <int NC_TAB, int NF>
__global__ void __launch_bounds__(PS_TPB) k_pairsum_multi_df(MultiArgs A, const float4* __restrict__ tab_g) {
    extern __shared__ float4 dtab[];
    __shared__ float4 txy[MDF_TILE];
    __shared__ float4 ts[MDF_TILE][MRB];
    const int words = A.ncell * (NC_TAB + 1) + (A.noct + 1) / 2;
    for (int i = threadIdx.x; i < words; i += PS_TPB) dtab[i] = tab_g[i];
    const float4* coef = dtab;
    const float4* cellv = dtab + (size_t)A.ncell * NC_TAB;
    const int2* oct = reinterpret_cast<const int2*>(cellv + A.ncell);
    const int n = A.n;
    const int j = blockIdx.x * PS_TPB + threadIdx.x;
    const int chunk = blockIdx.y;
    const int r0 = blockIdx.z * MRB;
    const int nr = min(MRB, A.R - r0);
    const int s_begin = chunk * A.spc;
    const int s_end = min(n, s_begin + A.spc);
    const double2 yj = A.xy[min(j, n - 1)];
    const DF tx = df_from(yj.x), ty = df_from(yj.y);
    double accr[MRB], acci[MRB];
#pragma unroll
    for (int q = 0; q < MRB; ++q) { accr[q] = 0.0; acci[q] = 0.0; }
    for (int base = s_begin; base < s_end; base += MDF_TILE) {
        __syncthreads();
        for (int i = threadIdx.x; i < MDF_TILE; i += PS_TPB) {
            const int src = base + i;
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
            if (src < s_end) {
                const double2 p = A.xy[src];
                const DF a = df_from(p.x), b = df_from(p.y);
                c = make_float4(a.h, a.l, b.h, b.l);
            }
            txy[i] = c;
        }
        for (int e = threadIdx.x; e < MDF_TILE * MRB; e += PS_TPB) {
            const int i = e / MRB, q = e % MRB, src = base + i;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (src < s_end && q < nr) {
                const double ww = A.w ? A.w[src] : 1.0;
                double2 ff = A.f[(size_t)(r0 + q) * A.sf + src];
                if (A.m) ff = cmul(A.m[src], ff);
                const DF re = df_from(ww * ff.x), im = df_from(ww * ff.y);
                v = make_float4(re.h, re.l, im.h, im.l);
            }
            ts[i][q] = v;
        }
        __syncthreads();
        float rh[MRB], rl[MRB], ih[MRB], il[MRB];
#pragma unroll
        for (int q = 0; q < MRB; ++q) { rh[q] = 0.f; rl[q] = 0.f; ih[q] = 0.f; il[q] = 0.f; }
        const int cnt = min(MDF_TILE, s_end - base);
        for (int i = 0; i < cnt; ++i) {
            DF hr, hi;
            if (!df_h0<NC_TAB, NF>(tx, ty, txy[i], coef, cellv, oct, A.noct, A.b_lo, A.k, A.inv_k, hr, hi)) continue;
#pragma unroll
            for (int q = 0; q < MRB; ++q) {
                const float4 sv = ts[i][q];
                // re += hr s_re - hi s_im, im += hr s_im + hi s_re
                const float p1 = hr.h * sv.x, p2 = hi.h * sv.z, p3 = hr.h * sv.z, p4 = hi.h * sv.x;
                float e1 = fmaf(hr.h, sv.x, -p1), e2 = fmaf(hi.h, sv.z, -p2);
                float e3 = fmaf(hr.h, sv.z, -p3), e4 = fmaf(hi.h, sv.x, -p4);
                e1 = fmaf(hr.l, sv.x, fmaf(hr.h, sv.y, e1));
                e2 = fmaf(hi.l, sv.z, fmaf(hi.h, sv.w, e2));
                e3 = fmaf(hr.l, sv.z, fmaf(hr.h, sv.w, e3));
                e4 = fmaf(hi.l, sv.x, fmaf(hi.h, sv.y, e4));
                float t, err;
                two_sum(rh[q], p1, t, err);
                rl[q] += err + e1;
                two_sum(t, -p2, rh[q], err);
                rl[q] += err - e2;
                two_sum(ih[q], p3, t, err);
                il[q] += err + e3;
                two_sum(t, p4, ih[q], err);
                il[q] += err + e4;
            }
        }
#pragma unroll
        for (int q = 0; q < MRB; ++q) {
            accr[q] += (double)rh[q] + (double)rl[q];
            acci[q] += (double)ih[q] + (double)il[q];
        }
    }
    if (j < n)
        for (int q = 0; q < nr; ++q)
            A.partial[((size_t)(r0 + q) * A.nchunk + chunk) * n + j] = make_double2(accr[q], acci[q]);
}

static void launch_multi_df(int nc, int nf, dim3 grid, size_t smem, cudaStream_t st, const MultiArgs& A,
                            const float4* tab) {
#define LS_MDF_LAUNCH(NC, NF) k_pairsum_multi_df<NC, NF><<<grid, PS_TPB, smem, st>>>(A, tab)
#define LS_MDF_NC(NC)                          \
    do {                                       \
        if (nf >= 4) LS_MDF_LAUNCH(NC, 4);     \
        else if (nf >= 2) LS_MDF_LAUNCH(NC, 2); \
        else LS_MDF_LAUNCH(NC, 0);             \
    } while (0)
    if (nc == 8) LS_MDF_NC(8);
    else if (nc == 9) LS_MDF_NC(9);
    else if (nc == 10) LS_MDF_NC(10);
    else LS_MDF_NC(12);
#undef LS_MDF_NC
#undef LS_MDF_LAUNCH
}

// Persistent form over several operators (scatterers): a block fetches work units
// (operator, target block, source chunk, RHS block) from an atomic counter until
// all units are done, reloading the shared-memory H0 table when the operator changes.
struct PSDesc {
    MultiArgs a;
    const float4* tab;
    int tab_words, tblocks, unit_begin, units;
};

__global__ void __launch_bounds__(PS_TPB) k_pairsum_persist(const PSDesc* __restrict__ d, int S, int total,
                                                            int* __restrict__ counter) {
    extern __shared__ float4 ftab[];
    __shared__ float4 txy[PS_TILE];
    __shared__ float2 ts[PS_TILE][MRB];
    __shared__ int s_unit;
    int cur = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_unit;
        if (u >= total) break;
        int s = 0;
        while (s + 1 < S && d[s + 1].unit_begin <= u) ++s;
        if (s != cur) {
            const float4* tg = d[s].tab;
            const int words = d[s].tab_words;
            for (int i = threadIdx.x; i < words; i += PS_TPB) ftab[i] = tg[i];
            cur = s;
            __syncthreads();
        }
        const int local = u - d[s].unit_begin;
        const int tb = local % d[s].tblocks;
        const int rest = local / d[s].tblocks;
        const int chunk = rest % d[s].a.nchunk;
        const int rb = rest / d[s].a.nchunk;
        multi_unit(d[s].a, tb, chunk, rb, ftab, txy, ts);
    }
}

#include "tc_pairsum.cuh"
#include "cr_solve.cuh"

// mode 0: y = x + k2 * ((i/4) sum_c partial + dV (m x));  mode 1: y = (i/4) sum_c partial
// partial[0][j] = sum over the slots of partial[c][j] (thread per node: every slot row is read
// coalesced), for the unordered-pair kernels' many slots; the epilogues then read one slot.
__global__ void k_sum_slots(int n, int nslots, double2* __restrict__ partial) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double sr = 0.0, si = 0.0;
#pragma unroll 8
    for (int c = 0; c < nslots; ++c) {
        const double2 p = partial[(size_t)c * n + j];
        sr += p.x;
        si += p.y;
    }
    partial[j] = make_double2(sr, si);
}

__global__ void k_apply_epi(int n, int nchunk, const double2* __restrict__ partial, const int64_t* __restrict__ rowptr,
                            const int* __restrict__ cols, const double2* __restrict__ vals,
                            const double2* __restrict__ m, const double2* __restrict__ x, double k2,
                            double2* __restrict__ y, int mode) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int j = warp;
    double sr = 0.0, si = 0.0;
    for (int c = lane; c < nchunk; c += 32) {
        double2 p = partial[(size_t)c * n + j];
        sr += p.x;
        si += p.y;
    }
    double cr = 0.0, ci = 0.0;
    if (mode == 0) {
        for (int64_t e = rowptr[j] + lane; e < rowptr[j + 1]; e += 32) {
            int q = cols[e];
            double2 f = cmul(m[q], x[q]);
            double2 t = cmul(vals[e], f);
            cr += t.x;
            ci += t.y;
        }
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    cr = warp_sum(cr);
    ci = warp_sum(ci);
    if (lane == 0) {
        // (i/4) (sr + i si) = (-si/4, sr/4)
        double vr = -0.25 * si, vi = 0.25 * sr;
        if (mode == 1) {
            y[j] = make_double2(vr, vi);
        } else {
            double2 xj = x[j];
            y[j] = make_double2(xj.x + k2 * (vr + cr), xj.y + k2 * (vi + ci));
        }
    }
}

// L^T x = x + k^2 m (w (i/4) sum_c partial + dV^T x), with the pair sum taken on unit
// weights (G is symmetric, so (K^T x)_n = w_n sum_j G(y_n, y_j) x_j).  mode 2 returns
// V^T x instead (no identity, no k^2 m factor).
__global__ void k_applyT_epi(int n, int nchunk, const double2* __restrict__ partial, const int64_t* __restrict__ rowptr,
                             const int* __restrict__ cols, const double2* __restrict__ vals,
                             const double2* __restrict__ m, const double* __restrict__ w,
                             const double2* __restrict__ x, double k2, double2* __restrict__ y, int mode) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int j = warp;
    double sr = 0.0, si = 0.0;
    for (int c = lane; c < nchunk; c += 32) {
        double2 p = partial[(size_t)c * n + j];
        sr += p.x;
        si += p.y;
    }
    double cr = 0.0, ci = 0.0;
    for (int64_t e = rowptr[j] + lane; e < rowptr[j + 1]; e += 32) {
        double2 t = cmul(vals[e], x[cols[e]]);
        cr += t.x;
        ci += t.y;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    cr = warp_sum(cr);
    ci = warp_sum(ci);
    if (lane == 0) {
        double2 vt = make_double2(w[j] * (-0.25 * si) + cr, w[j] * (0.25 * sr) + ci);   // (V^T x)_j
        if (mode == 2) {
            y[j] = vt;
        } else {
            double2 mv = cmul(m[j], vt);
            double2 xj = x[j];
            y[j] = make_double2(xj.x + k2 * mv.x, xj.y + k2 * mv.y);
        }
    }
}

// (A^T y)_l = sum_s A(l - s, l) y_{l - s} over grid rows l - s, A(j, j + s) = st[9 c(j) + s]
__global__ void k_stencilT(int nx, int ny, const double2* __restrict__ st, const double2* __restrict__ y,
                           const double2* __restrict__ g, double2* __restrict__ r) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nx * ny) return;
    int a = l % nx, b = l / nx;
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        int ja = a - (s % 3 - 1), jb = b - (s / 3 - 1);
        if (ja >= 0 && ja < nx && jb >= 0 && jb < ny)
            acc = cadd(acc, cmul(st[9 * grid_row_class(ja, jb, nx, ny) + s], y[ja + nx * jb]));
    }
    r[l] = csub(acc, g[l]);                  // (S^T - I) g = A^T C^{-T} g - g
}

// block transpose for the factors: out_b = in_b^T (row-major nx x nx blocks)
__global__ void k_transpose_blocks(int nx, int nblk, const double2* __restrict__ in, double2* __restrict__ out) {
    __shared__ double2 t[32][33];
    int b = blockIdx.z;
    if (b >= nblk) return;
    int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const double2* src = in + (size_t)b * nx * nx;
    double2* dst = out + (size_t)b * nx * nx;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        int r = y0 + i, c = x0 + threadIdx.x;
        if (r < nx && c < nx) t[i][threadIdx.x] = src[(size_t)r * nx + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        int r = x0 + i, c = y0 + threadIdx.x;
        if (r < nx && c < nx) dst[(size_t)r * nx + c] = t[threadIdx.x][i];
    }
}

// g_j = -k^2 e^{i pi/4}/sqrt(8 pi k) w_j sum_a conj(r_a) e^{-i k xhat_a . y_j}  (A^T conj(r))
__global__ void k_farfieldT(int n, const double2* __restrict__ xy, const double* __restrict__ w, double k, int n_ff,
                            const double* __restrict__ ang, const double2* __restrict__ r, double2* __restrict__ g) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double2 p = xy[j];
    double ar = 0.0, ai = 0.0;
    for (int a = 0; a < n_ff; ++a) {
        double cy, cx, s, c;
        sincos(ang[a], &cy, &cx);
        sincos(-k * fma(cx, p.x, cy * p.y), &s, &c);
        double2 rc = make_double2(r[a].x, -r[a].y);
        double2 t = cmul(rc, make_double2(c, s));
        ar += t.x;
        ai += t.y;
    }
    double gam = k * k / sqrt(8.0 * M_PI * k);
    double2 pre = make_double2(-gam * M_SQRT1_2 * w[j], -gam * M_SQRT1_2 * w[j]);
    g[j] = cmul(pre, make_double2(ar, ai));
}

// out = m * g (the adjoint right-hand side)
__global__ void k_cmul_vec(int n, const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = cmul(a[j], b[j]);
}

// grad_j += Re(u_j (g_j - k^2 vtl_j))
__global__ void k_grad_acc(int n, const double2* __restrict__ u, const double2* __restrict__ g,
                           const double2* __restrict__ vtl, double k2, double* __restrict__ grad) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double2 d = make_double2(g[j].x - k2 * vtl[j].x, g[j].y - k2 * vtl[j].y);
    grad[j] += u[j].x * d.x - u[j].y * d.y;
}

__global__ void k_hankel0(int64_t n, const double* __restrict__ z, double2* __restrict__ h) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) h[i] = ls_h0_r2(z[i] * z[i], 1.0, 1.0);
}

// ------------------------------------------------------------------ preconditioner apply
// g_i = sum_e tqc_vals[e] x[tqc_cols[e]]
__global__ void k_tqc(int nc, const int64_t* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ cv,
                      const double2* __restrict__ x, double2* __restrict__ g) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    double ar = 0.0, ai = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        double2 v = x[ci[e]];
        ar = fma(cv[e], v.x, ar);
        ai = fma(cv[e], v.y, ai);
    }
    g[i] = make_double2(ar, ai);
}

// t = A g: row (a, b) takes the stencil of its class over the in-grid offsets
__global__ void k_stencil(int nx, int ny, const double2* __restrict__ st, const double2* __restrict__ g,
                          double2* __restrict__ t) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nx * ny) return;
    int a = idx % nx, b = idx / nx;
    const double2* v = st + 9 * grid_row_class(a, b, nx, ny);
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        int la = a + s % 3 - 1, lb = b + s / 3 - 1;
        if (la >= 0 && la < nx && lb >= 0 && lb < ny) acc = cadd(acc, cmul(v[s], g[la + nx * lb]));
    }
    t[idx] = acc;
}

// z_q = w_q + sum_c psi_c (tp[i_c] - g[i_c])
__global__ void k_tcq(int nq, const int* __restrict__ idx, const double* __restrict__ wt, const double2* __restrict__ tp,
                      const double2* __restrict__ g, const double2* __restrict__ win, double2* __restrict__ z) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double2 acc = win[q];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int i = idx[4 * q + c];
        double2 d = g ? csub(tp[i], g[i]) : tp[i];
        acc.x = fma(wt[4 * q + c], d.x, acc.x);
        acc.y = fma(wt[4 * q + c], d.y, acc.y);
    }
    z[q] = acc;
}

// z_r[q] = x_r[q] + sum_e cv[e] t_r[ci[e]] over quadrature rows (the last step of P^T:
// x + (T_Q^C)^T r, any sparsity); grid.y = right-hand side r
__global__ void k_tqcT(int nq, const int64_t* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ cv,
                       const double2* __restrict__ t, size_t st, const double2* __restrict__ x, size_t sx,
                       double2* __restrict__ z, size_t sz) {
    const int r = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const double2* tr = t + (size_t)r * st;
    double2 acc = x[(size_t)r * sx + q];
    for (int64_t e = rp[q]; e < rp[q + 1]; ++e) {
        const double2 v = tr[ci[e]];
        acc.x = fma(cv[e], v.x, acc.x);
        acc.y = fma(cv[e], v.y, acc.y);
    }
    z[(size_t)r * sz + q] = acc;
}

// ------------------------------------------------------------------ block LU setup helpers
// S (column-major, nx x nx) = tri(Cd_b) - Cm_b * Gprev (Gprev row-major, may be null)
__global__ void k_build_S(int nx, int b, const double2* __restrict__ cband, const double2* __restrict__ Gprev,
                          double2* __restrict__ S) {
    int r = blockIdx.y;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx) return;
    const double2* base = cband + (size_t)b * 9 * nx;
    double2 v = make_double2(0.0, 0.0);
    int off = c - r;
    if (off >= -1 && off <= 1) v = base[(size_t)(3 + off + 1) * nx + r];     // db = 0 block, da = off
    if (Gprev) {
        for (int da = -1; da <= 1; ++da) {
            int t = r + da;
            if (t < 0 || t >= nx) continue;
            v = csub(v, cmul(base[(size_t)(da + 1) * nx + r], Gprev[(size_t)t * nx + c]));
        }
    }
    S[(size_t)c * nx + r] = v;
}

__global__ void k_identity_cm(int nx, double2* __restrict__ X) {
    int r = blockIdx.y;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nx) X[(size_t)c * nx + r] = make_double2(r == c ? 1.0 : 0.0, 0.0);
}

// W (row-major) = X (column-major);  G_b (row-major) = W_b Cp_b
__global__ void k_store_W_G(int nx, int b, int ny, const double2* __restrict__ X, const double2* __restrict__ cband,
                            double2* __restrict__ W, double2* __restrict__ Gm) {
    int r = blockIdx.y;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx) return;
    W[((size_t)b * nx + r) * nx + c] = X[(size_t)c * nx + r];
    if (b == ny - 1) return;
    const double2* Cp = cband + ((size_t)b * 9 + 6) * nx;    // db = +1 diagonals
    double2 acc = make_double2(0.0, 0.0);
    for (int da = -1; da <= 1; ++da) {                        // Cp(t, c) with c = t + da
        int t = c - da;
        if (t < 0 || t >= nx) continue;
        acc = cadd(acc, cmul(X[(size_t)t * nx + r], Cp[(size_t)(da + 1) * nx + t]));
    }
    Gm[((size_t)b * nx + r) * nx + c] = acc;
}

// ------------------------------------------------------------------ GMRES kernels
#define RED_TPB 256

// part[j * nblk + block] = sum_{rows of block} conj(V_j) z   for j < J
__global__ void k_dots(int n, int J, const double2* __restrict__ V, size_t ldv, const double2* __restrict__ z,
                       double2* __restrict__ part) {
    __shared__ double sr[RED_TPB / 32], si[RED_TPB / 32];
    const int nblk = gridDim.x;
    const int rows_per = (n + nblk - 1) / nblk;
    const int r0 = blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
    for (int j = 0; j < J; ++j) {
        const double2* v = V + (size_t)j * ldv;
        double ar = 0.0, ai = 0.0;
        for (int r = r0 + threadIdx.x; r < r1; r += RED_TPB) {
            double2 t = conjmul(v[r], z[r]);
            ar += t.x;
            ai += t.y;
        }
        ar = warp_sum(ar);
        ai = warp_sum(ai);
        if ((threadIdx.x & 31) == 0) { sr[threadIdx.x >> 5] = ar; si[threadIdx.x >> 5] = ai; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double tr = 0.0, ti = 0.0;
            for (int w = 0; w < RED_TPB / 32; ++w) { tr += sr[w]; ti += si[w]; }
            part[(size_t)j * nblk + blockIdx.x] = make_double2(tr, ti);
        }
        __syncthreads();
    }
}

// out[j] (+)= sum_b part[j * nblk + b]  (fixed order)
__global__ void k_sumrows(int J, int nblk, const double2* __restrict__ part, double2* __restrict__ out, int accumulate) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    double ar = 0.0, ai = 0.0;
    for (int b = 0; b < nblk; ++b) {
        double2 p = part[(size_t)j * nblk + b];
        ar += p.x;
        ai += p.y;
    }
    if (accumulate) { out[j].x += ar; out[j].y += ai; }
    else out[j] = make_double2(ar, ai);
}

// z -= sum_j V_j h_j
__global__ void k_update(int n, int J, const double2* __restrict__ V, size_t ldv, const double2* __restrict__ h,
                         double2* __restrict__ z) {
    extern __shared__ double2 hs[];
    for (int j = threadIdx.x; j < J; j += blockDim.x) hs[j] = h[j];
    __syncthreads();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double2 acc = z[r];
    for (int j = 0; j < J; ++j) {
        double2 t = cmul(V[(size_t)j * ldv + r], hs[j]);
        acc.x -= t.x;
        acc.y -= t.y;
    }
    z[r] = acc;
}

// u = sum_j V_j y_j
__global__ void k_combine(int n, int J, const double2* __restrict__ V, size_t ldv, const double2* __restrict__ yv,
                          double2* __restrict__ u) {
    extern __shared__ double2 ys[];
    for (int j = threadIdx.x; j < J; j += blockDim.x) ys[j] = yv[j];
    __syncthreads();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < J; ++j) acc = cadd(acc, cmul(V[(size_t)j * ldv + r], ys[j]));
    u[r] = acc;
}

// res = sqrt(nrm2_b) v0 - pu: the preconditioned residual P b - P L u from the first basis
// vector (P b / ||P b||) and the recombined operator products pu = sum_i y_i P L v_i
__global__ void k_resid_check(int n, const double2* __restrict__ v0, const double2* __restrict__ nrm2_b,
                              const double2* __restrict__ pu, double2* __restrict__ res) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const double beta = sqrt(nrm2_b->x);
    res[r] = make_double2(beta * v0[r].x - pu[r].x, beta * v0[r].y - pu[r].y);
}

// y = a - b
__global__ void k_sub_vec(int n, const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ y) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) y[r] = csub(a[r], b[r]);
}

// J = 1/2 sum |uinf - t|^2 over total entries (one block, fixed order); resid = uinf - t
__global__ void k_misfit(int total, const double2* __restrict__ uinf, const double2* __restrict__ t,
                         double2* __restrict__ resid, double* __restrict__ J) {
    __shared__ double part[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const double2 d = csub(uinf[i], t[i]);
        resid[i] = d;
        acc = fma(d.x, d.x, fma(d.y, d.y, acc));
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *J = 0.5 * part[0];
}

// w = w' / D
__global__ void k_div_real(int n, const double* __restrict__ D, double2* __restrict__ w) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) w[r] = make_double2(w[r].x / D[r], w[r].y / D[r]);
}

// rho = sum_j D_j conj(Sw_j) w_j / sum_j D_j |w_j|^2 (one block, fixed order)
__global__ void k_rho(int n, const double* __restrict__ D, const double2* __restrict__ w, const double2* __restrict__ Sw,
                      double* __restrict__ out) {
    __shared__ double pr[256], pi[256], pd[256];
    double ar = 0.0, ai = 0.0, ad = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double2 t = conjmul(Sw[j], w[j]);
        ar = fma(D[j], t.x, ar);
        ai = fma(D[j], t.y, ai);
        ad = fma(D[j], w[j].x * w[j].x + w[j].y * w[j].y, ad);
    }
    pr[threadIdx.x] = ar; pi[threadIdx.x] = ai; pd[threadIdx.x] = ad;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            pr[threadIdx.x] += pr[threadIdx.x + o];
            pi[threadIdx.x] += pi[threadIdx.x + o];
            pd[threadIdx.x] += pd[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = pr[0] / pd[0]; out[1] = pi[0] / pd[0]; }
}

// m = Re(m_real) + 0 i from a real device vector
__global__ void k_real_to_complex(int n, const double* __restrict__ a, double2* __restrict__ out) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) out[r] = make_double2(a[r], 0.0);
}

// dst = src / nrm (nrm = sqrt(*nrm2)); writes nrm to *hout if given
__global__ void k_scale(int n, const double2* __restrict__ src, const double2* __restrict__ nrm2, double2* __restrict__ dst,
                        double2* hout) {
    double nr = sqrt(nrm2->x);
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0 && hout) *hout = make_double2(nr, 0.0);
    if (r >= n) return;
    double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    double2 v = src[r];
    dst[r] = make_double2(v.x * inv, v.y * inv);
}

// Givens update of Hessenberg column j (column-major, leading dimension ldh)
__global__ void k_givens(int j, double2* H, int ldh, double2* cs, double2* sn, double2* g, double* hist,
                         const double2* beta2) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2* col = H + (size_t)j * ldh;
    for (int i = 0; i < j; ++i) {
        double2 a = col[i], b = col[i + 1];
        double2 t = cadd(cmul(cs[i], a), cmul(sn[i], b));
        double2 cc = make_double2(cs[i].x, -cs[i].y), sc = make_double2(sn[i].x, -sn[i].y);
        col[i + 1] = csub(cmul(cc, b), cmul(sc, a));
        col[i] = t;
    }
    double2 a = col[j], b = col[j + 1];
    double den = sqrt(a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y);
    double2 c, s;
    if (den > 0.0) {
        c = make_double2(a.x / den, -a.y / den);
        s = make_double2(b.x / den, -b.y / den);
    } else {
        c = make_double2(1.0, 0.0);
        s = make_double2(0.0, 0.0);
    }
    cs[j] = c;
    sn[j] = s;
    col[j] = make_double2(den, 0.0);
    col[j + 1] = make_double2(0.0, 0.0);
    double2 gj = g[j];
    double2 sc = make_double2(s.x, -s.y);
    double2 gn = cmul(sc, gj);
    g[j + 1] = make_double2(-gn.x, -gn.y);
    g[j] = cmul(c, gj);
    double beta = sqrt(beta2->x);
    hist[j + 1] = sqrt(g[j + 1].x * g[j + 1].x + g[j + 1].y * g[j + 1].y) / beta;
}

// y = H(0:it, 0:it)^{-1} g(0:it) (upper triangular)
__global__ void k_backsolve(int it, const double2* H, int ldh, const double2* g, double2* yv) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = it - 1; i >= 0; --i) {
        double2 acc = g[i];
        for (int c = i + 1; c < it; ++c) acc = csub(acc, cmul(H[(size_t)c * ldh + i], yv[c]));
        double2 d = H[(size_t)i * ldh + i];
        double dd = d.x * d.x + d.y * d.y;
        yv[i] = make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
    }
}

__global__ void k_gmres_init(double2* g, const double2* beta2, double* hist) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        g[0] = make_double2(sqrt(beta2->x), 0.0);
        hist[0] = 1.0;
    }
}

// ------------------------------------------------------------------ batched (R systems, blockIdx.y = r)
// Vectors of system r live at base + r * stride.
__global__ void k_apply_epi_multi(int n, int nchunk, const double2* __restrict__ partial, const int64_t* __restrict__ rowptr,
                                  const int* __restrict__ cols, const double2* __restrict__ vals,
                                  const double2* __restrict__ m, const double2* __restrict__ x, size_t sx, double k2,
                                  double2* __restrict__ y, size_t sy) {
    const int r = blockIdx.y;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int j = warp;
    const double2* xr = x + (size_t)r * sx;
    const double2* pr = partial + (size_t)r * nchunk * n;
    double sr = 0.0, si = 0.0;
    for (int c = lane; c < nchunk; c += 32) {
        double2 p = pr[(size_t)c * n + j];
        sr += p.x;
        si += p.y;
    }
    double cr = 0.0, ci = 0.0;
    for (int64_t e = rowptr[j] + lane; e < rowptr[j + 1]; e += 32) {
        int q = cols[e];
        double2 t = cmul(vals[e], cmul(m[q], xr[q]));
        cr += t.x;
        ci += t.y;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    cr = warp_sum(cr);
    ci = warp_sum(ci);
    if (lane == 0) {
        double2 xj = xr[j];
        y[(size_t)r * sy + j] = make_double2(xj.x + k2 * (-0.25 * si + cr), xj.y + k2 * (0.25 * sr + ci));
    }
}

__global__ void k_tqc_multi(int nc, const int64_t* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ cv,
                            const double2* __restrict__ x, size_t sx, double2* __restrict__ g) {
    int r = blockIdx.y;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double2* xr = x + (size_t)r * sx;
    double ar = 0.0, ai = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        double2 v = xr[ci[e]];
        ar = fma(cv[e], v.x, ar);
        ai = fma(cv[e], v.y, ai);
    }
    g[(size_t)r * nc + i] = make_double2(ar, ai);
}

__global__ void k_stencil_multi(int nx, int ny, const double2* __restrict__ st, const double2* __restrict__ g,
                                double2* __restrict__ t) {
    int r = blockIdx.y;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int nc = nx * ny;
    if (idx >= nc) return;
    const double2* gr = g + (size_t)r * nc;
    int a = idx % nx, b = idx / nx;
    const double2* v = st + 9 * grid_row_class(a, b, nx, ny);
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        int la = a + s % 3 - 1, lb = b + s / 3 - 1;
        if (la >= 0 && la < nx && lb >= 0 && lb < ny) acc = cadd(acc, cmul(v[s], gr[la + nx * lb]));
    }
    t[(size_t)r * nc + idx] = acc;
}

__global__ void k_bt_fwd_multi(int nx, int ny, int b, const double2* __restrict__ W, const double2* __restrict__ cband,
                               const double2* __restrict__ t, double2* __restrict__ y) {
    extern __shared__ double2 sh[];
    const int r = blockIdx.y;
    const size_t off = (size_t)r * nx * ny;
    const double2* Cm = cband + (size_t)b * 9 * nx;
    for (int c = threadIdx.x; c < nx; c += blockDim.x) {
        double2 v = t[off + (size_t)b * nx + c];
        if (b > 0) {
            const double2* yp = y + off + (size_t)(b - 1) * nx;
            for (int da = -1; da <= 1; ++da) {
                int cc = c + da;
                if (cc >= 0 && cc < nx) v = csub(v, cmul(Cm[(size_t)(da + 1) * nx + c], yp[cc]));
            }
        }
        sh[c] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= nx) return;
    const double2* Wr = W + ((size_t)b * nx + row) * nx;
    double ar = 0.0, ai = 0.0;
    for (int c = lane; c < nx; c += 32) {
        double2 wv = Wr[c], v = sh[c];
        ar = fma(wv.x, v.x, fma(-wv.y, v.y, ar));
        ai = fma(wv.x, v.y, fma(wv.y, v.x, ai));
    }
    ar = warp_sum(ar);
    ai = warp_sum(ai);
    if (lane == 0) y[off + (size_t)b * nx + row] = make_double2(ar, ai);
}

__global__ void k_bt_bwd_multi(int nx, int ny, int b, const double2* __restrict__ Gm, double2* __restrict__ y) {
    extern __shared__ double2 sh[];
    const size_t off = (size_t)blockIdx.y * nx * ny;
    for (int c = threadIdx.x; c < nx; c += blockDim.x) sh[c] = y[off + (size_t)(b + 1) * nx + c];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= nx) return;
    const double2* Gr = Gm + ((size_t)b * nx + row) * nx;
    double ar = 0.0, ai = 0.0;
    for (int c = lane; c < nx; c += 32) {
        double2 gv = Gr[c], v = sh[c];
        ar = fma(gv.x, v.x, fma(-gv.y, v.y, ar));
        ai = fma(gv.x, v.y, fma(gv.y, v.x, ai));
    }
    ar = warp_sum(ar);
    ai = warp_sum(ai);
    if (lane == 0) {
        double2 v = y[off + (size_t)b * nx + row];
        y[off + (size_t)b * nx + row] = make_double2(v.x - ar, v.y - ai);
    }
}

// Batched block-LU sweeps of C in FP32 (used by the tensor-core batched form, which refines
// its solutions against an accurate residual, so the preconditioner only has to be close):
// one launch per block row b; a CTA computes a tile of BT_ROWS rows x BT_RHS right-hand
// sides of
//   forward   y_b = W_b (t_b - L_b y_{b-1})       (L_b: the 3-point lower band of C)
//   backward  y_b = y_b - G_b y_{b+1}
// staging BT_KC columns of the factor and of the input vectors in shared memory per step,
// with the K = nx reduction split over the 8 warps and summed in shared memory at the end.
// Thread (lane) computes rows 4 rg .. 4 rg + 3 (rg = lane / 4) x RHS 2 rq, 2 rq + 1 (rq = lane % 4).
#define BT_ROWS 32
#define BT_RHS 8
#define BT_KC 64
__global__ void __launch_bounds__(256) k_bt_sweep32(int nx, int ny, int b, int R, int backward,
                                                    const float2* __restrict__ M, const float2* __restrict__ cb,
                                                    const double2* __restrict__ t, float2* __restrict__ y) {
    __shared__ float2 Ws[BT_ROWS][BT_KC + 1];
    __shared__ __align__(16) float2 Vs[BT_KC][BT_RHS];
    __shared__ float2 red[8][BT_ROWS * BT_RHS];
    const int row0 = blockIdx.x * BT_ROWS, rhs0 = blockIdx.y * BT_RHS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rg = lane >> 2, rq = lane & 3;
    const size_t plane = (size_t)nx * ny;
    const float2* Mb = M + (size_t)b * nx * nx;
    float ar[4][2], ai[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q) ar[i][q] = ai[i][q] = 0.f;
    for (int k0 = 0; k0 < nx; k0 += BT_KC) {
        __syncthreads();
        for (int i = threadIdx.x; i < BT_ROWS * BT_KC; i += blockDim.x) {
            const int r = i / BT_KC, kk = i % BT_KC, row = row0 + r, k = k0 + kk;
            Ws[r][kk] = (row < nx && k < nx) ? Mb[(size_t)row * nx + k] : make_float2(0.f, 0.f);
        }
        for (int i = threadIdx.x; i < BT_KC * BT_RHS; i += blockDim.x) {
            const int kk = i % BT_KC, q = i / BT_KC, k = k0 + kk, r = rhs0 + q;
            float2 v = make_float2(0.f, 0.f);
            if (k < nx && r < R) {
                const size_t o = (size_t)r * plane;
                if (backward) {
                    v = y[o + (size_t)(b + 1) * nx + k];
                } else {
                    const double2 tv = t[o + (size_t)b * nx + k];
                    v = make_float2((float)tv.x, (float)tv.y);
                    if (b > 0) {
                        const float2* cbb = cb + (size_t)b * 9 * nx;
                        const float2* yp = y + o + (size_t)(b - 1) * nx;
#pragma unroll
                        for (int da = -1; da <= 1; ++da) {
                            const int kc = k + da;
                            if (kc >= 0 && kc < nx) {
                                const float2 c = cbb[(size_t)(da + 1) * nx + k], yv = yp[kc];
                                v.x -= fmaf(c.x, yv.x, -c.y * yv.y);
                                v.y -= fmaf(c.x, yv.y, c.y * yv.x);
                            }
                        }
                    }
                }
            }
            Vs[kk][q] = v;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < BT_KC / 8; ++j) {
            const int kk = warp * (BT_KC / 8) + j;
            const float4 vv = *reinterpret_cast<const float4*>(&Vs[kk][2 * rq]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 w = Ws[4 * rg + i][kk];
                ar[i][0] = fmaf(w.x, vv.x, fmaf(-w.y, vv.y, ar[i][0]));
                ai[i][0] = fmaf(w.x, vv.y, fmaf(w.y, vv.x, ai[i][0]));
                ar[i][1] = fmaf(w.x, vv.z, fmaf(-w.y, vv.w, ar[i][1]));
                ai[i][1] = fmaf(w.x, vv.w, fmaf(w.y, vv.z, ai[i][1]));
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 2; ++q) red[warp][(4 * rg + i) * BT_RHS + 2 * rq + q] = make_float2(ar[i][q], ai[i][q]);
    __syncthreads();
    for (int o = threadIdx.x; o < BT_ROWS * BT_RHS; o += blockDim.x) {
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            sr += red[w][o].x;
            si += red[w][o].y;
        }
        const int row = row0 + o / BT_RHS, rhs = rhs0 + o % BT_RHS;
        if (row < nx && rhs < R) {
            float2* yo = y + (size_t)rhs * plane + (size_t)b * nx + row;
            if (backward) {
                const float2 v = *yo;
                *yo = make_float2(v.x - sr, v.y - si);
            } else {
                *yo = make_float2(sr, si);
            }
        }
    }
}

__global__ void k_to_f32(int64_t n, const double2* __restrict__ a, float2* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

__global__ void k_to_f64(int64_t n, const float2* __restrict__ a, double2* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_double2((double)a[i].x, (double)a[i].y);
}

__global__ void k_tcq_multi(int nq, int nc, const int* __restrict__ idx, const double* __restrict__ wt,
                            const double2* __restrict__ tp, const double2* __restrict__ g, const double2* __restrict__ win,
                            size_t sin_, double2* __restrict__ z, size_t sz) {
    int r = blockIdx.y;
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const double2* tpr = tp + (size_t)r * nc;
    const double2* gr = g ? g + (size_t)r * nc : nullptr;
    double2 acc = win[(size_t)r * sin_ + q];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int i = idx[4 * q + c];
        double2 d = g ? csub(tpr[i], gr[i]) : tpr[i];
        acc.x = fma(wt[4 * q + c], d.x, acc.x);
        acc.y = fma(wt[4 * q + c], d.y, acc.y);
    }
    z[(size_t)r * sz + q] = acc;
}

// part[(r * J + j) * nblk + block] = conj(V_{r,j}) . z_r over the block's rows
__global__ void k_dots_multi(int n, int J, const double2* __restrict__ V, size_t sv_r, size_t ldv,
                             const double2* __restrict__ z, size_t sz, double2* __restrict__ part, const int* __restrict__ active) {
    __shared__ double sr[RED_TPB / 32], si[RED_TPB / 32];
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    const int nblk = gridDim.x;
    const int rows_per = (n + nblk - 1) / nblk;
    const int r0 = blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
    const double2* zr = z + (size_t)r * sz;
    for (int j = 0; j < J; ++j) {
        const double2* v = V + (size_t)r * sv_r + (size_t)j * ldv;
        double ar = 0.0, ai = 0.0;
        for (int q = r0 + threadIdx.x; q < r1; q += RED_TPB) {
            double2 t = conjmul(v[q], zr[q]);
            ar += t.x;
            ai += t.y;
        }
        ar = warp_sum(ar);
        ai = warp_sum(ai);
        if ((threadIdx.x & 31) == 0) { sr[threadIdx.x >> 5] = ar; si[threadIdx.x >> 5] = ai; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double tr = 0.0, ti = 0.0;
            for (int w = 0; w < RED_TPB / 32; ++w) { tr += sr[w]; ti += si[w]; }
            part[((size_t)r * J + j) * nblk + blockIdx.x] = make_double2(tr, ti);
        }
        __syncthreads();
    }
}

// out[r * so + j] (+)= sum_b part[(r * J + j) * nblk + b]
__global__ void k_sumrows_multi(int J, int nblk, const double2* __restrict__ part, double2* __restrict__ out, size_t so,
                                int accumulate, const int* __restrict__ active) {
    int r = blockIdx.y;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J || (active && !active[r])) return;
    double ar = 0.0, ai = 0.0;
    for (int b = 0; b < nblk; ++b) {
        double2 p = part[((size_t)r * J + j) * nblk + b];
        ar += p.x;
        ai += p.y;
    }
    double2* o = out + (size_t)r * so + j;
    if (accumulate) { o->x += ar; o->y += ai; }
    else *o = make_double2(ar, ai);
}

__global__ void k_update_multi(int n, int J, const double2* __restrict__ V, size_t sv_r, size_t ldv,
                               const double2* __restrict__ h, size_t sh_r, double2* __restrict__ z, size_t sz,
                               const int* __restrict__ active) {
    extern __shared__ double2 hs[];
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    for (int j = threadIdx.x; j < J; j += blockDim.x) hs[j] = h[(size_t)r * sh_r + j];
    __syncthreads();
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    double2* zr = z + (size_t)r * sz;
    double2 acc = zr[q];
    for (int j = 0; j < J; ++j) {
        double2 t = cmul(V[(size_t)r * sv_r + (size_t)j * ldv + q], hs[j]);
        acc.x -= t.x;
        acc.y -= t.y;
    }
    zr[q] = acc;
}

// dst_r = src_r / sqrt(nrm2[r].x); hout[r * sh] = the norm
__global__ void k_scale_multi(int n, const double2* __restrict__ src, size_t ss, const double2* __restrict__ nrm2,
                              double2* __restrict__ dst, size_t sd, double2* hout, size_t sh, const int* __restrict__ active) {
    const int r = blockIdx.y;
    if (active && !active[r]) return;
    double nr = sqrt(nrm2[r].x);
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0 && hout) hout[(size_t)r * sh] = make_double2(nr, 0.0);
    if (q >= n) return;
    double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    double2 v = src[(size_t)r * ss + q];
    dst[(size_t)r * sd + q] = make_double2(v.x * inv, v.y * inv);
}

// one thread per system: Givens update of column j; deactivates converged systems
__global__ void k_givens_multi(int R, int j, double2* H, size_t sH, int ldh, double2* cs, double2* sn, double2* g,
                               size_t sg, double* hist, size_t shist, const double2* beta2, double tol, int* active,
                               int* its) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R || !active[r]) return;
    double2* col = H + (size_t)r * sH + (size_t)j * ldh;
    double2* csr = cs + (size_t)r * sg;
    double2* snr = sn + (size_t)r * sg;
    double2* gr = g + (size_t)r * sg;
    for (int i = 0; i < j; ++i) {
        double2 a = col[i], b = col[i + 1];
        double2 t = cadd(cmul(csr[i], a), cmul(snr[i], b));
        double2 cc = make_double2(csr[i].x, -csr[i].y), sc = make_double2(snr[i].x, -snr[i].y);
        col[i + 1] = csub(cmul(cc, b), cmul(sc, a));
        col[i] = t;
    }
    double2 a = col[j], b = col[j + 1];
    double den = sqrt(a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y);
    double2 c = den > 0.0 ? make_double2(a.x / den, -a.y / den) : make_double2(1.0, 0.0);
    double2 s_ = den > 0.0 ? make_double2(b.x / den, -b.y / den) : make_double2(0.0, 0.0);
    csr[j] = c;
    snr[j] = s_;
    col[j] = make_double2(den, 0.0);
    col[j + 1] = make_double2(0.0, 0.0);
    double2 gj = gr[j];
    double2 gn = cmul(make_double2(s_.x, -s_.y), gj);
    gr[j + 1] = make_double2(-gn.x, -gn.y);
    gr[j] = cmul(c, gj);
    double res = sqrt(gr[j + 1].x * gr[j + 1].x + gr[j + 1].y * gr[j + 1].y) / sqrt(beta2[r].x);
    hist[(size_t)r * shist + j + 1] = res;
    its[r] = j + 1;
    if (!(res > tol)) active[r] = 0;
}

__global__ void k_backsolve_multi(int R, const int* its, const double2* H, size_t sH, int ldh, const double2* g, size_t sg,
                                  double2* yv, size_t sy) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    int it = its[r];
    const double2* Hr = H + (size_t)r * sH;
    const double2* gr = g + (size_t)r * sg;
    double2* yr = yv + (size_t)r * sy;
    for (int i = it - 1; i >= 0; --i) {
        double2 acc = gr[i];
        for (int c = i + 1; c < it; ++c) acc = csub(acc, cmul(Hr[(size_t)c * ldh + i], yr[c]));
        double2 d = Hr[(size_t)i * ldh + i];
        double dd = d.x * d.x + d.y * d.y;
        yr[i] = make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
    }
}

__global__ void k_combine_multi(int n, const int* its, const double2* __restrict__ V, size_t sv_r, size_t ldv,
                                const double2* __restrict__ yv, size_t sy, double2* __restrict__ u, size_t su) {
    const int r = blockIdx.y;
    const int it = its[r];
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < it; ++j) acc = cadd(acc, cmul(V[(size_t)r * sv_r + (size_t)j * ldv + q], yv[(size_t)r * sy + j]));
    u[(size_t)r * su + q] = acc;
}

// batched L^T epilogue: y_r = x_r + k^2 m (w (i/4) sum_c partial_r + dV^T x_r)
__global__ void k_applyT_epi_multi(int n, int nchunk, const double2* __restrict__ partial, const int64_t* __restrict__ rowptr,
                                   const int* __restrict__ cols, const double2* __restrict__ vals,
                                   const double2* __restrict__ m, const double* __restrict__ w,
                                   const double2* __restrict__ x, size_t sx, double k2, double2* __restrict__ y, size_t sy) {
    const int r = blockIdx.y;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int j = warp;
    const double2* xr = x + (size_t)r * sx;
    const double2* pr = partial + (size_t)r * nchunk * n;
    double sr = 0.0, si = 0.0;
    for (int c = lane; c < nchunk; c += 32) {
        double2 p = pr[(size_t)c * n + j];
        sr += p.x;
        si += p.y;
    }
    double cr = 0.0, ci = 0.0;
    for (int64_t e = rowptr[j] + lane; e < rowptr[j + 1]; e += 32) {
        double2 t = cmul(vals[e], xr[cols[e]]);
        cr += t.x;
        ci += t.y;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    cr = warp_sum(cr);
    ci = warp_sum(ci);
    if (lane == 0) {
        double2 vt = make_double2(w[j] * (-0.25 * si) + cr, w[j] * (0.25 * sr) + ci);
        if (!m) {                                   // V^T x alone
            y[(size_t)r * sy + j] = vt;
            return;
        }
        double2 mv = cmul(m[j], vt);
        double2 xj = xr[j];
        y[(size_t)r * sy + j] = make_double2(xj.x + k2 * mv.x, xj.y + k2 * mv.y);
    }
}

__global__ void k_btT_fwd_multi(int nx, int ny, int b, const double2* __restrict__ GT, double2* __restrict__ z) {
    extern __shared__ double2 sh[];
    const size_t off = (size_t)blockIdx.y * nx * ny;
    for (int c = threadIdx.x; c < nx; c += blockDim.x) sh[c] = z[off + (size_t)(b - 1) * nx + c];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= nx) return;
    const double2* Gr = GT + ((size_t)(b - 1) * nx + row) * nx;
    double ar = 0.0, ai = 0.0;
    for (int c = lane; c < nx; c += 32) {
        double2 gv = Gr[c], v = sh[c];
        ar = fma(gv.x, v.x, fma(-gv.y, v.y, ar));
        ai = fma(gv.x, v.y, fma(gv.y, v.x, ai));
    }
    ar = warp_sum(ar);
    ai = warp_sum(ai);
    if (lane == 0) {
        double2 v = z[off + (size_t)b * nx + row];
        z[off + (size_t)b * nx + row] = make_double2(v.x - ar, v.y - ai);
    }
}

__global__ void k_btT_bwd_multi(int nx, int ny, int b, const double2* __restrict__ WT, const double2* __restrict__ cband,
                                const double2* __restrict__ z, double2* __restrict__ x) {
    extern __shared__ double2 sh[];
    const size_t off = (size_t)blockIdx.y * nx * ny;
    for (int c = threadIdx.x; c < nx; c += blockDim.x) {
        double2 v = z[off + (size_t)b * nx + c];
        if (b + 1 < ny) {
            const double2* Cm1 = cband + (size_t)(b + 1) * 9 * nx;
            const double2* xn = x + off + (size_t)(b + 1) * nx;
            for (int da = -1; da <= 1; ++da) {
                int a = c - da;
                if (a >= 0 && a < nx) v = csub(v, cmul(Cm1[(size_t)(da + 1) * nx + a], xn[a]));
            }
        }
        sh[c] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= nx) return;
    const double2* Wr = WT + ((size_t)b * nx + row) * nx;
    double ar = 0.0, ai = 0.0;
    for (int c = lane; c < nx; c += 32) {
        double2 wv = Wr[c], v = sh[c];
        ar = fma(wv.x, v.x, fma(-wv.y, v.y, ar));
        ai = fma(wv.x, v.y, fma(wv.y, v.x, ai));
    }
    ar = warp_sum(ar);
    ai = warp_sum(ai);
    if (lane == 0) x[off + (size_t)b * nx + row] = make_double2(ar, ai);
}

__global__ void k_stencilT_multi(int nx, int ny, const double2* __restrict__ st, const double2* __restrict__ y,
                                 const double2* __restrict__ g, double2* __restrict__ r) {
    const int nc = nx * ny;
    const size_t off = (size_t)blockIdx.y * nc;
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nc) return;
    int a = l % nx, b = l / nx;
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        int ja = a - (s % 3 - 1), jb = b - (s / 3 - 1);
        if (ja >= 0 && ja < nx && jb >= 0 && jb < ny)
            acc = cadd(acc, cmul(st[9 * grid_row_class(ja, jb, nx, ny) + s], y[off + ja + nx * jb]));
    }
    r[off + l] = csub(acc, g[off + l]);
}

// r_r = b_r - y_r and u_r += d_r over R systems of n entries (contiguous rows)
__global__ void k_residual_multi(int64_t total, const double2* __restrict__ b, const double2* __restrict__ y,
                                 double2* __restrict__ r) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) r[i] = csub(b[i], y[i]);
}

__global__ void k_accumulate_multi(int64_t total, const double2* __restrict__ d, double2* __restrict__ u) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) u[i] = cadd(u[i], d[i]);
}

__global__ void k_gmres_init_multi(int R, double2* g, size_t sg, const double2* beta2, double* hist, size_t shist, int* active,
                                   int* its) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    its[r] = 0;
    g[(size_t)r * sg] = make_double2(sqrt(beta2[r].x), 0.0);
    hist[(size_t)r * shist] = 1.0;
    active[r] = beta2[r].x > 0.0 ? 1 : 0;
}

// ------------------------------------------------------------------ outputs
__global__ void k_incident(int n, const double2* __restrict__ xy, double k, double dx, double dy, double2* __restrict__ b) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double2 p = xy[j];
    double s, c;
    sincos(k * fma(dx, p.x, dy * p.y), &s, &c);
    b[j] = make_double2(c, s);
}

__global__ void k_farfield(int n, const double2* __restrict__ xy, const double* __restrict__ w,
                           const double2* __restrict__ m, const double2* __restrict__ u, double k,
                           const double* __restrict__ ang, double2* __restrict__ out) {
    __shared__ double sr[RED_TPB / 32], si[RED_TPB / 32];
    double th = ang[blockIdx.x];
    double cx, cy;
    sincos(th, &cy, &cx);
    double ar = 0.0, ai = 0.0;
    for (int j = threadIdx.x; j < n; j += RED_TPB) {
        double2 p = xy[j];
        double s, c;
        sincos(-k * fma(cx, p.x, cy * p.y), &s, &c);
        double2 f = cmul(m[j], u[j]);
        double2 t = cmul(f, make_double2(c, s));
        ar = fma(w[j], t.x, ar);
        ai = fma(w[j], t.y, ai);
    }
    ar = warp_sum(ar);
    ai = warp_sum(ai);
    if ((threadIdx.x & 31) == 0) { sr[threadIdx.x >> 5] = ar; si[threadIdx.x >> 5] = ai; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0, ti = 0.0;
        for (int q = 0; q < RED_TPB / 32; ++q) { tr += sr[q]; ti += si[q]; }
        // -k^2 e^{i pi/4} / sqrt(8 pi k)
        double gam = k * k / sqrt(8.0 * M_PI * k);
        double2 pre = make_double2(-gam * M_SQRT1_2, -gam * M_SQRT1_2);
        out[blockIdx.x] = cmul(pre, make_double2(tr, ti));
    }
}

// FP64 FMA-rate probe: 8 independent dependent chains per thread
__global__ void k_probe_dfma(int iters, double a, double b, double* sink) {
    double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    double s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == 123.456) sink[0] = s;
}

// ------------------------------------------------------------------ host structures
struct ls_mesh {
    HostMesh h;
};

template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t count) {
        if (p) { cudaFree(p); p = nullptr; }
        n = count;
        if (count == 0) return cudaSuccess;
        return cudaMalloc(&p, count * sizeof(T));
    }
};

// Cyclic-reduction solve of C (cr_solve.cuh): persistent factor blocks, the vector
// arena [t | x | scratch] and the launch steps of C x = t and C^T x = t.
struct CRPlan {
    struct Step { int kind; int first; int count; };   // kind 0: dense products, 1: band, 2: band transposed
    int nx = 0, ny = 0;
    size_t svec = 0;                                    // arena stride per right-hand side
    DevBuf<double2> store, arena;
    DevBuf<CRJob> jobs;
    DevBuf<CRTriJob> tjobs;
    std::vector<Step> fwd, trn;
    std::vector<CRJob> hjobs;                           // host copy of jobs (for the double-float variant)
    DevBuf<float4> store_df;                            // store as double-float pairs (made on first use)
    DevBuf<CRJobDF> jobs_df;
    double2* t() const { return arena.p; }
    double2* x() const { return arena.p + (size_t)nx * ny; }
};

struct ls_op {
    int nq = 0;
    double k = 0;
    ls_params prm{};
    cudaStream_t stream = nullptr;
    // mesh and operator data
    DevBuf<double2> xy, m;
    DevBuf<double> w;
    DevBuf<int64_t> rowptr, rowptrT;
    DevBuf<int> cols, colsT;
    DevBuf<double2> vals, valsT;         // dV and its transpose
    CsrC host_csr;
    std::vector<double> host_nodes, host_w;
    // pair-sum decomposition and scratch
    int nchunk = 1, src_per_chunk = 0;
    DevBuf<double2> partial;
    int ps_slots = 1;                    // partial rows written by the last single-RHS pair sum
    // symmetric double-float pair sum (k_pairsum_dfs): blocks, distance chunks, distances per chunk
    bool df_sym = true;
    int dfs_nb = 1, dfs_nchunk = 1, dfs_dper = 1;
    // tabulated H0 (pairsum mode 0: FP64 table, mode 2: FP32 table, modes 3 and 4: double-float
    // table; mode 4 also keeps the FP32 table tab32 for its inner solves)
    int mode = 0;
    bool use_table = false;
    int tab_nc = 12;                     // table degree + 1 chosen by the setup autotuner
    int tab_nf = 0;                      // double-float form: top coefficients summed in FP32
    bool inner32 = false;                // mixed form (mode 4): pair sums of the inner solves in FP32
    float tune_ms[4] = {0, 0, 0, 0};     // pair-sum time of the NC = 12, 10, 9 (, 8) candidates (0: not tried)
    int tab_ncell = 0, tab_noct = 0, tab_blo = 0;
    size_t tab_bytes = 0;
    double tab_err = 0, tab_tlo = 0, tab_thi = 0;
    DevBuf<double2> tab;
    // preconditioner
    bool has_prec = false;
    int nx = 0, ny = 0;
    DevBuf<int> tcq_idx;
    DevBuf<double> tcq_w;
    DevBuf<int64_t> tqc_rp;
    DevBuf<int> tqc_ci;
    DevBuf<double> tqc_cv;
    DevBuf<double2> cband, Wf, Gf;
    DevBuf<double2> WT, GT;              // transposed factors for P^T
    DevBuf<float2> Wf32, Gf32, cband32, by32;   // FP32 copies for the tensor-core batched sweeps
    DevBuf<int64_t> tcqT_rp, tqcT_rp;    // (T_C^Q)^T over grid rows, (T_Q^C)^T over quadrature rows (for P^T)
    DevBuf<int> tcqT_ci, tqcT_ci;
    DevBuf<double> tcqT_cv, tqcT_cv;
    int n_interior = 0;                  // grid nodes inside the mesh (Approach I) or pixelation nodes (II)
    DevBuf<double> Dg;                   // Approach II column sums D (1 off the pixelation), Eq. D_def
    DevBuf<double2> st;                  // [9 classes][9 offsets] sparsifying stencils
    DevBuf<double2> pg, pt, ptp;         // grid work vectors
    // GMRES workspace
    DevBuf<double2> Vb, H, cs, sn, g, hv, yv, tmp, tmp2, dpart, scal;
    DevBuf<double2> Wb;                  // raw operator products P L v_j of the last solve (exit check)
    DevBuf<double2> Hraw;                // Hessenberg matrix of the last solve before the Givens rotations
    int last_it = 0;                     // iterations of the last single-RHS GMRES solve
    double last_res = -1.0;              // explicit relative residual of the last single-RHS solve(s) (max)
    DevBuf<double> hist;
    int dblk = 0;
    // batched form: FP32 table and lock-step GMRES workspace for R systems
    DevBuf<double2> tab32;
    int t32_ncell = 0, t32_noct = 0, t32_blo = 0;
    size_t t32_bytes = 0;
    int bR = 0, b_nchunk = 1, b_spc = 0;
    int b_nchunk_cur = 1;                // chunk count of the partials written by the last batched pair sum
    // batched pair sum on the tensor cores (k_pairsum_tc): split densities, coordinates, error word
    int batch_kernel = 1;                // 0: CUDA cores (k_pairsum_multi_f32), 1: tensor cores
    int tc_fold = 4;                     // stages per accumulator run
    int tc_refine = 4;                   // iterative-refinement steps after a tensor-core solve (0: none)
    bool refine_single = false;          // refinement residuals from an FP64-accurate operator
    bool refine_user = false;            // refine_single set by ls_op_set_batch_refine (else: follows the form)
    uint64_t tc_stall_ns = 0;            // failure-detection test: forced stall of the MMA issuer (ns)
    int64_t corr_host_blocks = 0;        // correction blocks the device setup left to the host
    DevBuf<double2> ir_r, ir_d, ir_y;    // refinement work vectors [R][n]
    int tc_nchunk = 0, tc_spc = 0, tc_npad = 0;
    DevBuf<float4> tc_xy32, tc_Sc;
    DevBuf<int> tc_err;
    DevBuf<TCOp> tc_desc;                // per-launch operator descriptors (up to TC_MAX_OPS)
    std::vector<TCOp> tc_hdesc;
    int* tc_herr = nullptr;              // pinned copy of tc_err
    DevBuf<double2> bV, bH, bcs, bsn, bg, bhv, byv, btmp, bdpart, bscal, bpartial, bpg, bpt, bptp;
    DevBuf<double> bhist;
    DevBuf<int> bactive, bits;
    // setup phase times (s): correction, grid transfers + stencil + C, block LU, H0 table
    double t_setup[4] = {0, 0, 0, 0};
    // CUDA graph of the preconditioner apply (fixed input/output buffers)
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gP = nullptr;
    DevBuf<double2> pin, pout;
    cudaGraphExec_t gPT = nullptr;         // graph of the P^T apply
    cudaGraphExec_t gPdf = nullptr, gPTdf = nullptr;   // the same with the double-float blocks
    int nlaunch_P = 0, nlaunch_PT = 0;     // kernels in each graph
    int nlaunch_Pdf = 0, nlaunch_PTdf = 0;
    CRPlan cr;                           // cyclic reduction of C for the single-RHS P and P^T
    // purely Cartesian operator (ls_cartesian_create): the unknowns are the grid nodes,
    // L^(C) = I + k^2 V^(C) M^(C) with V^(C) applied by FFT convolution, P = S^(C) = C^{-1} A
    bool cartesian = false;
    int cNX = 0, cNY = 0;                // zero-padded FFT grid (2 nx x 2 ny)
    cufftHandle fft = 0;
    DevBuf<double2> khat, fpad, czero;   // kernel spectrum / (NX NY), padded work array, zeros
    // instrumentation: kernel launches on this operator, CUDA-event timing of the pair sum
    int64_t launches = 0, pairsum_launches = 0;
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    std::vector<int8_t> ev_kind;         // arithmetic of each timed launch (LS_PREC_*; 10/11 batched kernels)
    ~ls_op() {
        for (auto& e : ev) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
        if (gP) cudaGraphExecDestroy(gP);
        if (gPT) cudaGraphExecDestroy(gPT);
        if (gPdf) cudaGraphExecDestroy(gPdf);
        if (gPTdf) cudaGraphExecDestroy(gPTdf);
        if (cap) cudaStreamDestroy(cap);
        if (tc_herr) cudaFreeHost(tc_herr);
        if (fft) cufftDestroy(fft);
    }
};

static ls_status check_stream_sync(ls_op* op) {
    CK(cudaStreamSynchronize(op->stream));
    CK(cudaGetLastError());
    return LS_OK;
}

// ------------------------------------------------------------------ building blocks
static void launch_tab(int nc, dim3 grid, size_t smem, cudaStream_t st, const double2* xy, const double* w,
                       const double2* m, const double2* f, int n, int spc, double k, const double2* tab, int ncell,
                       int noct, int blo, double2* partial) {
    const double ik = 1.0 / k;
    if (nc == 9) k_pairsum_tab<9><<<grid, PS_TPB, smem, st>>>(xy, w, m, f, n, spc, k, ik, tab, ncell, noct, blo, partial);
    else if (nc == 10) k_pairsum_tab<10><<<grid, PS_TPB, smem, st>>>(xy, w, m, f, n, spc, k, ik, tab, ncell, noct, blo, partial);
    else k_pairsum_tab<12><<<grid, PS_TPB, smem, st>>>(xy, w, m, f, n, spc, k, ik, tab, ncell, noct, blo, partial);
}

static void launch_df(int nc, int nf, dim3 grid, size_t smem, cudaStream_t st, const double2* xy, const double* w,
                      const double2* m, const double2* f, int n, int spc, double k, const float4* tab, int ncell,
                      int noct, int blo, double2* partial) {
    const double ik = 1.0 / k;
#define LS_DF_LAUNCH(NC, NF) k_pairsum_df<NC, NF><<<grid, PS_TPB, smem, st>>>(xy, w, m, f, n, spc, k, ik, tab, ncell, noct, blo, partial)
#define LS_DF_NC(NC)                          \
    do {                                      \
        if (nf >= 4) LS_DF_LAUNCH(NC, 4);     \
        else if (nf >= 2) LS_DF_LAUNCH(NC, 2); \
        else LS_DF_LAUNCH(NC, 0);             \
    } while (0)
    if (nc == 8) LS_DF_NC(8);
    else if (nc == 9) LS_DF_NC(9);
    else if (nc == 10) LS_DF_NC(10);
    else LS_DF_NC(12);
#undef LS_DF_NC
#undef LS_DF_LAUNCH
}

static void launch_dfs(int nc, int nf, dim3 grid, size_t smem, cudaStream_t st, const double2* xy, const double* w,
                       const double2* m, const double2* f, int n, int nb, int dper, double k, const float4* tab,
                       int ncell, int noct, int blo, double2* partial) {
    const double ik = 1.0 / k;
#define LS_DFS_LAUNCH(NC, NF) \
    k_pairsum_dfs<NC, NF><<<grid, PS_TPB, smem, st>>>(xy, w, m, f, n, nb, dper, k, ik, tab, ncell, noct, blo, partial)
#define LS_DFS_NC(NC)                          \
    do {                                       \
        if (nf >= 4) LS_DFS_LAUNCH(NC, 4);     \
        else if (nf >= 2) LS_DFS_LAUNCH(NC, 2); \
        else LS_DFS_LAUNCH(NC, 0);             \
    } while (0)
    if (nc == 8) LS_DFS_NC(8);
    else if (nc == 9) LS_DFS_NC(9);
    else if (nc == 10) LS_DFS_NC(10);
    else LS_DFS_NC(12);
#undef LS_DFS_NC
#undef LS_DFS_LAUNCH
}

static cudaError_t raise_tab_limits(int mode, size_t bytes) {
    cudaError_t e = cudaSuccess;
    if (mode == 3) {
#define LS_DF_RAISE(NC)                                                                        \
        if ((e = raise_smem_limit(k_pairsum_df<NC, 0>, bytes)) != cudaSuccess) return e;      \
        if ((e = raise_smem_limit(k_pairsum_df<NC, 2>, bytes)) != cudaSuccess) return e;      \
        if ((e = raise_smem_limit(k_pairsum_df<NC, 4>, bytes)) != cudaSuccess) return e;      \
        if ((e = raise_smem_limit(k_pairsum_dfs<NC, 0>, bytes)) != cudaSuccess) return e;     \
        if ((e = raise_smem_limit(k_pairsum_dfs<NC, 2>, bytes)) != cudaSuccess) return e;     \
        if ((e = raise_smem_limit(k_pairsum_dfs<NC, 4>, bytes)) != cudaSuccess) return e;     \
        if ((e = raise_smem_limit(k_pairsum_multi_df<NC, 0>, bytes)) != cudaSuccess) return e; \
        if ((e = raise_smem_limit(k_pairsum_multi_df<NC, 2>, bytes)) != cudaSuccess) return e; \
        if ((e = raise_smem_limit(k_pairsum_multi_df<NC, 4>, bytes)) != cudaSuccess) return e;
        LS_DF_RAISE(8)
        LS_DF_RAISE(9)
        LS_DF_RAISE(10)
        LS_DF_RAISE(12)
#undef LS_DF_RAISE
        return cudaSuccess;
    }
    if ((e = raise_smem_limit(k_pairsum_tab<9>, bytes)) != cudaSuccess) return e;
    if ((e = raise_smem_limit(k_pairsum_tab<10>, bytes)) != cudaSuccess) return e;
    return raise_smem_limit(k_pairsum_tab<12>, bytes);
}

static ls_status launch_pairsum(ls_op* op, const double2* f, const double2* m, const double* w);
static ls_status launch_pairsum(ls_op* op, const double2* f, const double2* m) { return launch_pairsum(op, f, m, op->w.p); }

// Many partial slots (the unordered-pair kernels): sum them into slot 0 with coalesced reads
// before the epilogue, which then reads one slot.
static ls_status collapse_slots(ls_op* op) {
    if (op->ps_slots <= 32) return LS_OK;
    k_sum_slots<<<(op->nq + 255) / 256, 256, 0, op->stream>>>(op->nq, op->ps_slots, op->partial.p);
    CK(cudaGetLastError());
    op->launches++;
    op->ps_slots = 1;
    return LS_OK;
}

static ls_status launch_pairsum(ls_op* op, const double2* f, const double2* m, const double* w) {
    if (op->cartesian) return fail(LS_EINVAL, "a purely Cartesian operator has no quadrature-node pair sum");
    dim3 grid((op->nq + PS_TPB - 1) / PS_TPB, op->nchunk);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (op->timing && op->ev.size() < 65536) {
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        op->ev.emplace_back(e0, e1);
        op->ev_kind.push_back((int8_t)(op->mode == 4 ? (op->inner32 ? 2 : 3) : op->mode));
        CK(cudaEventRecord(e0, op->stream));
    }
    op->ps_slots = op->nchunk;
    const bool df = op->mode == 3 || (op->mode == 4 && !op->inner32);
    if (df && op->df_sym) {
        const int D = op->dfs_nb / 2;
        op->ps_slots = op->dfs_nchunk + D;
        if (D > 0 && 2 * D == op->dfs_nb)      // slot of distance nb / 2: half of it stays unwritten
            CK(cudaMemsetAsync(op->partial.p + (size_t)(op->ps_slots - 1) * op->nq, 0, sizeof(double2) * op->nq,
                               op->stream));
        launch_dfs(op->tab_nc, op->tab_nf, dim3(op->dfs_nb, op->dfs_nchunk), op->tab_bytes, op->stream, op->xy.p, w, m,
                   f, op->nq, op->dfs_nb, op->dfs_dper, op->k, (const float4*)op->tab.p, op->tab_ncell, op->tab_noct,
                   op->tab_blo, op->partial.p);
    } else if (df)
        launch_df(op->tab_nc, op->tab_nf, grid, op->tab_bytes, op->stream, op->xy.p, w, m, f, op->nq, op->src_per_chunk, op->k,
                  (const float4*)op->tab.p, op->tab_ncell, op->tab_noct, op->tab_blo, op->partial.p);
    else if (op->mode == 2 || op->mode == 4) {
        // FP32 table: the operator's own (mode 2) or the mixed form's inner one (mode 4)
        const bool inner = op->mode == 4;
        const size_t bytes = inner ? op->t32_bytes : op->tab_bytes;
        const float4* tab = (const float4*)(inner ? op->tab32.p : op->tab.p);
        const int ncell = inner ? op->t32_ncell : op->tab_ncell, noct = inner ? op->t32_noct : op->tab_noct;
        const int blo = inner ? op->t32_blo : op->tab_blo;
        if (op->df_sym) {
            const int D = op->dfs_nb / 2;
            op->ps_slots = op->dfs_nchunk + D;
            if (D > 0 && 2 * D == op->dfs_nb)
                CK(cudaMemsetAsync(op->partial.p + (size_t)(op->ps_slots - 1) * op->nq, 0, sizeof(double2) * op->nq,
                                   op->stream));
            k_pairsum_f32s<<<dim3(op->dfs_nb, op->dfs_nchunk), PS_TPB, bytes, op->stream>>>(
                op->xy.p, w, m, f, op->nq, op->dfs_nb, op->dfs_dper, op->k, 1.0 / op->k, tab, ncell, noct, blo,
                op->partial.p);
        } else {
            k_pairsum_f32<<<grid, PS_TPB, bytes, op->stream>>>(op->xy.p, w, m, f, op->nq, op->src_per_chunk, op->k,
                                                               1.0 / op->k, tab, ncell, noct, blo, op->partial.p);
        }
    }
    else if (op->use_table)
        launch_tab(op->tab_nc, grid, op->tab_bytes, op->stream, op->xy.p, w, m, f, op->nq, op->src_per_chunk, op->k,
                   op->tab.p, op->tab_ncell, op->tab_noct, op->tab_blo, op->partial.p);
    else
        k_pairsum<<<grid, PS_TPB, 0, op->stream>>>(op->xy.p, w, m, f, op->nq, op->src_per_chunk, op->k, 1.0 / op->k,
                                                   op->partial.p);
    CK(cudaGetLastError());
    if (e1) CK(cudaEventRecord(e1, op->stream));
    op->launches++;
    op->pairsum_launches++;
    return LS_OK;
}

// ------------------------------------------------------------------ purely Cartesian operator
// padded input: f[b][a] = (m x)_(a, b) (or x when m is null) inside the nx x ny block, 0 elsewhere
__global__ void k_cart_pad(int nx, int ny, int NX, int NY, const double2* __restrict__ m, const double2* __restrict__ x,
                           double2* __restrict__ f) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (a >= NX || b >= NY) return;
    double2 v = make_double2(0.0, 0.0);
    if (a < nx && b < ny) {
        const int j = a + nx * b;
        v = m ? cmul(m[j], x[j]) : x[j];
    }
    f[(size_t)b * NX + a] = v;
}

__global__ void k_cart_mul(int64_t n, const double2* __restrict__ khat, double2* __restrict__ f) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i] = cmul(khat[i], f[i]);
}

// mode 0: y = x + k2 V(m x);  mode 1: y = x + k2 m V(x);  mode 2: y = V(x)
__global__ void k_cart_epi(int nx, int ny, int NX, const double2* __restrict__ x, const double2* __restrict__ m,
                           const double2* __restrict__ f, double k2, double2* __restrict__ y, int mode) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (a >= nx || b >= ny) return;
    const int j = a + nx * b;
    const double2 v = f[(size_t)b * NX + a];
    if (mode == 2) { y[j] = v; return; }
    const double2 w = mode == 1 ? cmul(m[j], v) : v;
    y[j] = make_double2(x[j].x + k2 * w.x, x[j].y + k2 * w.y);
}

// padded kernel K(da, db) from the table of offsets (|da|, |db|) (V^(C) is even in both)
__global__ void k_cart_kernel(int nx, int ny, int NX, int NY, const double2* __restrict__ tab, double2* __restrict__ K) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (a >= NX || b >= NY) return;
    const int da = a < nx ? a : NX - a, db = b < ny ? b : NY - b;   // offsets 0..nx-1 and -(nx-1)..-1
    double2 v = make_double2(0.0, 0.0);
    if (da < nx && db < ny && a != nx && b != ny) v = tab[(size_t)db * nx + da];
    K[(size_t)b * NX + a] = v;
}

static ls_status cart_apply(ls_op* op, const double2* x, double2* y, int mode) {
    const int nx = op->nx, ny = op->ny, NX = op->cNX, NY = op->cNY;
    dim3 gp((NX + 127) / 128, NY), ge((nx + 127) / 128, ny);
    k_cart_pad<<<gp, 128, 0, op->stream>>>(nx, ny, NX, NY, mode == 0 ? op->m.p : nullptr, x, op->fpad.p);
    if (cufftExecZ2Z(op->fft, (cufftDoubleComplex*)op->fpad.p, (cufftDoubleComplex*)op->fpad.p, CUFFT_FORWARD) !=
        CUFFT_SUCCESS)
        return fail(LS_ECUDA, "cufftExecZ2Z (forward) failed");
    const int64_t tot = (int64_t)NX * NY;
    k_cart_mul<<<(unsigned)((tot + 255) / 256), 256, 0, op->stream>>>(tot, op->khat.p, op->fpad.p);
    if (cufftExecZ2Z(op->fft, (cufftDoubleComplex*)op->fpad.p, (cufftDoubleComplex*)op->fpad.p, CUFFT_INVERSE) !=
        CUFFT_SUCCESS)
        return fail(LS_ECUDA, "cufftExecZ2Z (inverse) failed");
    k_cart_epi<<<ge, 128, 0, op->stream>>>(nx, ny, NX, x, op->m.p, op->fpad.p, op->k * op->k, y, mode);
    CK(cudaGetLastError());
    op->launches += 3;
    return LS_OK;
}

static ls_status apply_L(ls_op* op, const double2* x, double2* y) {
    if (op->cartesian) return cart_apply(op, x, y, 0);
    ls_status s = launch_pairsum(op, x, op->m.p);
    if (s != LS_OK) return s;
    TRY(collapse_slots(op));
    int threads = 256;
    int blocks = (int)(((int64_t)op->nq * 32 + threads - 1) / threads);
    k_apply_epi<<<blocks, threads, 0, op->stream>>>(op->nq, op->ps_slots, op->partial.p, op->rowptr.p, op->cols.p, op->vals.p,
                                                    op->m.p, x, op->k * op->k, y, 0);
    CK(cudaGetLastError());
    op->launches++;
    return LS_OK;
}

// ------------------------------------------------------------------ cyclic reduction (host)
#define CKB(call)                                                                                 \
    do {                                                                                          \
        cublasStatus_t s_ = (call);                                                               \
        if (s_ != CUBLAS_STATUS_SUCCESS)                                                          \
            return fail(LS_ECUDA, std::string(#call) + ": cublas status " + std::to_string(s_));  \
    } while (0)

// Batched row-major products C_b = alpha A_b B_b + beta C_b (cuBLAS is column-major:
// a row-major matrix is its transpose there, so the operands are passed swapped).
static ls_status cr_gemm(cublasHandle_t h, cudaStream_t st, int nx, double alpha, double beta,
                         const std::vector<const double2*>& A, const std::vector<const double2*>& B,
                         const std::vector<double2*>& C, DevBuf<const double2*>& scratch) {
    const int cnt = (int)C.size();
    if (cnt == 0) return LS_OK;
    std::vector<const double2*> ptrs(3 * (size_t)cnt);
    for (int i = 0; i < cnt; ++i) { ptrs[i] = B[i]; ptrs[cnt + i] = A[i]; ptrs[2 * cnt + i] = C[i]; }
    CK(scratch.alloc(ptrs.size()));
    CK(cudaMemcpyAsync(scratch.p, ptrs.data(), sizeof(void*) * ptrs.size(), cudaMemcpyHostToDevice, st));
    const cuDoubleComplex a = make_cuDoubleComplex(alpha, 0.0), b = make_cuDoubleComplex(beta, 0.0);
    CKB(cublasZgemmBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, nx, nx, nx, &a, (const cuDoubleComplex* const*)scratch.p, nx,
                           (const cuDoubleComplex* const*)(scratch.p + cnt), nx, &b,
                           (cuDoubleComplex* const*)(scratch.p + 2 * cnt), nx, cnt));
    CK(cudaStreamSynchronize(st));            // the pointer scratch is reused by the next call
    return LS_OK;
}

// Factor blocks of the cyclic reduction of C (cr_solve.cuh) and the job tables of
// both solves.  Needs op->cband, op->nx, op->ny.
static ls_status build_cr(ls_op* op) {
    CRPlan& P = op->cr;
    const int nx = op->nx, ny = op->ny;
    const size_t bs = (size_t)nx * nx, nc = (size_t)nx * ny;
    cudaStream_t st = op->stream;
    P.nx = nx;
    P.ny = ny;
    std::vector<int> nl{ny};
    while (nl.back() > 1) nl.push_back((nl.back() + 1) / 2);
    const int NL = (int)nl.size() - 1;                 // levels with an elimination
    const size_t NONE = SIZE_MAX;
    // persistent slots (in blocks): per level the odd rows' Dinv, gamma, delta and, from
    // level 1 on, every row's L and U; the transposed copy of slot s is slot s + nN
    std::vector<std::vector<size_t>> sDinv(NL), sGam(NL), sDlt(NL), sL(NL + 1), sU(NL + 1);
    size_t nN = 0;
    for (int l = 0; l < NL; ++l) {
        const int n = nl[l];
        for (int i = 1; i < n; i += 2) {
            sDinv[l].push_back(nN++);
            sGam[l].push_back(nN++);
            sDlt[l].push_back(i + 1 < n ? nN++ : NONE);
        }
        const int n1 = nl[l + 1];
        sL[l + 1].assign(n1, NONE);
        sU[l + 1].assign(n1, NONE);
        if (n1 > 1)
            for (int p = 0; p < n1; ++p) {
                if (p >= 1) sL[l + 1][p] = nN++;
                if (2 * p + 2 < n) sU[l + 1][p] = nN++;
            }
    }
    const size_t sTop = nN++;
    CK(P.store.alloc(2 * nN * bs));
    auto blk = [&](size_t s) { return P.store.p + s * bs; };
    // working blocks: D of every row (updated in place level by level), dense level-0 L and U
    DevBuf<double2> work;
    CK(work.alloc(3 * (size_t)ny * bs));
    double2* Dw = work.p;
    double2* L0 = work.p + (size_t)ny * bs;
    double2* U0 = work.p + 2 * (size_t)ny * bs;
    {
        std::vector<int> ids(ny);
        std::vector<double2*> outD(ny), outL(ny), outU(ny);
        for (int b = 0; b < ny; ++b) {
            ids[b] = b;
            outD[b] = Dw + b * bs;
            outL[b] = L0 + b * bs;
            outU[b] = U0 + b * bs;
        }
        DevBuf<int> dids;
        DevBuf<double2*> dout;
        CK(dids.alloc(ny));
        CK(dout.alloc(3 * (size_t)ny));
        CK(cudaMemcpy(dids.p, ids.data(), sizeof(int) * ny, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dout.p, outL.data(), sizeof(void*) * ny, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dout.p + ny, outD.data(), sizeof(void*) * ny, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dout.p + 2 * ny, outU.data(), sizeof(void*) * ny, cudaMemcpyHostToDevice));
        for (int which = 0; which < 3; ++which) {
            dim3 g((nx + 127) / 128, nx, ny);
            k_cr_expand<<<g, 128, 0, st>>>(nx, op->cband.p, dids.p, which, dout.p + (size_t)which * ny);
        }
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
    }
    // current level's blocks (null: no such coupling)
    std::vector<double2*> Dp(ny), Lp(ny), Up(ny);
    for (int b = 0; b < ny; ++b) {
        Dp[b] = Dw + b * bs;
        Lp[b] = b > 0 ? L0 + b * bs : nullptr;
        Up[b] = b + 1 < ny ? U0 + b * bs : nullptr;
    }
    cusolverDnHandle_t hs = nullptr;
    CKS(cusolverDnCreate(&hs));
    struct HS { cusolverDnHandle_t h; ~HS() { cusolverDnDestroy(h); } } gs{hs};
    CKS(cusolverDnSetStream(hs, st));
    cublasHandle_t hb = nullptr;
    CKB(cublasCreate(&hb));
    struct HB { cublasHandle_t h; ~HB() { cublasDestroy(h); } } gb{hb};
    CKB(cublasSetStream(hb, st));
    int lwork = 0;
    CKS(cusolverDnZgetrf_bufferSize(hs, nx, nx, (cuDoubleComplex*)Dw, nx, &lwork));
    DevBuf<double2> wsp;
    DevBuf<int> piv, info;
    CK(wsp.alloc(std::max(lwork, 1)));
    CK(piv.alloc(nx));
    CK(info.alloc((size_t)ny + 1));
    CK(cudaMemsetAsync(info.p, 0, sizeof(int) * (ny + 1), st));
    DevBuf<const double2*> pscr;
    DevBuf<double2*> tptr;
    CK(tptr.alloc(1));
    int ninv = 0;
    // X = D^{-1} (row-major) by LU of the column-major view D^T: X^T = (D^T)^{-1}
    auto invert = [&](double2* D, double2* X) -> ls_status {
        CK(cudaMemcpyAsync(tptr.p, &X, sizeof(void*), cudaMemcpyHostToDevice, st));
        k_cr_identity<<<dim3((nx + 127) / 128, nx, 1), 128, 0, st>>>(nx, tptr.p);
        CK(cudaGetLastError());
        CKS(cusolverDnZgetrf(hs, nx, nx, (cuDoubleComplex*)D, nx, (cuDoubleComplex*)wsp.p, piv.p, info.p + ninv));
        CKS(cusolverDnZgetrs(hs, CUBLAS_OP_N, nx, nx, (const cuDoubleComplex*)D, nx, piv.p, (cuDoubleComplex*)X, nx,
                             info.p + ny));
        CK(cudaStreamSynchronize(st));        // tptr is reused
        ++ninv;
        return LS_OK;
    };
    for (int l = 0; l < NL; ++l) {
        const int n = nl[l];
        std::vector<const double2*> A, B;
        std::vector<double2*> C;
        for (int i = 1, o = 0; i < n; i += 2, ++o) TRY(invert(Dp[i], blk(sDinv[l][o])));
        for (int i = 1, o = 0; i < n; i += 2, ++o) {            // gamma_i = Dinv_i L_i, delta_i = Dinv_i U_i
            A.push_back(blk(sDinv[l][o])); B.push_back(Lp[i]); C.push_back(blk(sGam[l][o]));
            if (sDlt[l][o] != NONE) { A.push_back(blk(sDinv[l][o])); B.push_back(Up[i]); C.push_back(blk(sDlt[l][o])); }
        }
        TRY(cr_gemm(hb, st, nx, 1.0, 0.0, A, B, C, pscr));
        A.clear(); B.clear(); C.clear();
        for (int j = 2; j < n; j += 2) {                           // D_j -= L_j delta_{j-1}
            A.push_back(Lp[j]); B.push_back(blk(sDlt[l][(j - 1) / 2])); C.push_back(Dp[j]);
        }
        TRY(cr_gemm(hb, st, nx, -1.0, 1.0, A, B, C, pscr));
        A.clear(); B.clear(); C.clear();
        for (int j = 0; j + 1 < n; j += 2) {                       // D_j -= U_j gamma_{j+1}
            A.push_back(Up[j]); B.push_back(blk(sGam[l][j / 2])); C.push_back(Dp[j]);
        }
        TRY(cr_gemm(hb, st, nx, -1.0, 1.0, A, B, C, pscr));
        A.clear(); B.clear(); C.clear();
        const int n1 = nl[l + 1];
        if (n1 > 1) {
            for (int p = 0; p < n1; ++p) {
                const int j = 2 * p;
                if (sL[l + 1][p] != NONE) { A.push_back(Lp[j]); B.push_back(blk(sGam[l][(j - 1) / 2])); C.push_back(blk(sL[l + 1][p])); }
                if (sU[l + 1][p] != NONE) { A.push_back(Up[j]); B.push_back(blk(sDlt[l][(j + 1) / 2])); C.push_back(blk(sU[l + 1][p])); }
            }
            TRY(cr_gemm(hb, st, nx, -1.0, 0.0, A, B, C, pscr));
        }
        std::vector<double2*> D2(n1), L2(n1), U2(n1);
        for (int p = 0; p < n1; ++p) {
            D2[p] = Dp[2 * p];
            L2[p] = sL[l + 1][p] != NONE ? blk(sL[l + 1][p]) : nullptr;
            U2[p] = sU[l + 1][p] != NONE ? blk(sU[l + 1][p]) : nullptr;
        }
        Dp.swap(D2); Lp.swap(L2); Up.swap(U2);
    }
    TRY(invert(Dp[0], blk(sTop)));
    {
        std::vector<int> hinfo(ny + 1);
        CK(cudaMemcpy(hinfo.data(), info.p, sizeof(int) * (ny + 1), cudaMemcpyDeviceToHost));
        for (int i = 0; i <= ny; ++i)
            if (hinfo[i] != 0) return fail(LS_ESINGULAR, "cyclic reduction: a diagonal block of C is singular");
    }
    {   // transposed copies
        std::vector<const double2*> in(nN);
        std::vector<double2*> out(nN);
        for (size_t s = 0; s < nN; ++s) { in[s] = blk(s); out[s] = blk(s + nN); }
        DevBuf<const double2*> din;
        DevBuf<double2*> dout;
        CK(din.alloc(nN));
        CK(dout.alloc(nN));
        CK(cudaMemcpy(din.p, in.data(), sizeof(void*) * nN, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dout.p, out.data(), sizeof(void*) * nN, cudaMemcpyHostToDevice));
        for (size_t s0 = 0; s0 < nN; s0 += 65535) {
            const unsigned cnt = (unsigned)std::min<size_t>(65535, nN - s0);
            dim3 tb(32, 8), tg((nx + 31) / 32, (nx + 31) / 32, cnt);
            k_cr_transpose<<<tg, tb, 0, st>>>(nx, din.p + s0, dout.p + s0);
        }
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
    }
    // vector arena [t | x | scratch] and the job tables; scratch: per level the z of the
    // odd rows and the right-hand side of the next level
    size_t nscr = 0;
    for (int l = 0; l < NL; ++l) nscr += (size_t)(nl[l] / 2) + (size_t)nl[l + 1];
    CK(P.arena.alloc(2 * nc + nscr * nx));
    P.svec = 2 * nc + nscr * nx;
    double2* scr = P.arena.p + 2 * nc;
    size_t soff = 0;
    auto take = [&]() { double2* p = scr + soff; soff += nx; return p; };
    std::vector<std::vector<double2*>> T(NL + 1), Z(NL);
    T[0].resize(ny);
    for (int b = 0; b < ny; ++b) T[0][b] = P.t() + (size_t)b * nx;
    for (int l = 0; l < NL; ++l) {
        for (int i = 1; i < nl[l]; i += 2) Z[l].push_back(take());
        for (int p = 0; p < nl[l + 1]; ++p) T[l + 1].push_back(take());
    }
    if (soff > nscr * nx) return fail(LS_ECUDA, "cyclic reduction: scratch overflow");
    auto X = [&](int l, int p) { return P.x() + ((size_t)p << l) * nx; };
    auto N_ = [&](size_t s) -> const double2* { return s == NONE ? nullptr : blk(s); };
    auto T_ = [&](size_t s) -> const double2* { return s == NONE ? nullptr : blk(s + nN); };
    std::vector<CRJob> J;
    std::vector<CRTriJob> TJ;
    auto dense = [&](double2* y, const double2* base, const double2* M1, const double2* v1, const double2* M2,
                     const double2* v2) {
        if (!M1) { M1 = M2; v1 = v2; M2 = nullptr; v2 = nullptr; }
        J.push_back(CRJob{y, base, M1, v1, M2, M2 ? v2 : nullptr});
    };
    auto step = [&](std::vector<CRPlan::Step>& list, int kind, size_t first) {
        const size_t cnt = (kind == 0 ? J.size() : TJ.size()) - first;
        if (cnt) list.push_back({kind, (int)first, (int)cnt});
    };
    // C x = t
    for (int l = 0; l < NL; ++l) {
        const int n = nl[l];
        size_t f0 = J.size();
        for (int i = 1, o = 0; i < n; i += 2, ++o) dense(Z[l][o], nullptr, N_(sDinv[l][o]), T[l][i], nullptr, nullptr);
        step(P.fwd, 0, f0);
        if (l == 0) {
            size_t t0 = TJ.size();
            for (int j = 0; j < n; j += 2)
                TJ.push_back(CRTriJob{T[1][j / 2], T[0][j], j >= 1 ? Z[0][(j - 1) / 2] : nullptr,
                                      j + 1 < n ? Z[0][(j + 1) / 2] : nullptr, j >= 1 ? j : -1, j + 1 < n ? j : -1});
            step(P.fwd, 1, t0);
        } else {
            f0 = J.size();
            for (int j = 0; j < n; j += 2)
                dense(T[l + 1][j / 2], T[l][j], j >= 1 ? N_(sL[l][j]) : nullptr, j >= 1 ? Z[l][(j - 1) / 2] : nullptr,
                      j + 1 < n ? N_(sU[l][j]) : nullptr, j + 1 < n ? Z[l][(j + 1) / 2] : nullptr);
            step(P.fwd, 0, f0);
        }
    }
    {
        size_t f0 = J.size();
        dense(X(NL, 0), nullptr, N_(sTop), T[NL][0], nullptr, nullptr);
        step(P.fwd, 0, f0);
    }
    for (int l = NL - 1; l >= 0; --l) {
        const int n = nl[l];
        size_t f0 = J.size();
        for (int i = 1, o = 0; i < n; i += 2, ++o)
            dense(X(l, i), Z[l][o], N_(sGam[l][o]), X(l, i - 1), N_(sDlt[l][o]), i + 1 < n ? X(l, i + 1) : nullptr);
        step(P.fwd, 0, f0);
    }
    // C^T x = t
    for (int l = 0; l < NL; ++l) {
        const int n = nl[l];
        size_t f0 = J.size();
        for (int j = 0; j < n; j += 2)
            dense(T[l + 1][j / 2], T[l][j], j + 1 < n ? T_(sGam[l][j / 2]) : nullptr, j + 1 < n ? T[l][j + 1] : nullptr,
                  j >= 1 ? T_(sDlt[l][(j - 1) / 2]) : nullptr, j >= 1 ? T[l][j - 1] : nullptr);
        step(P.trn, 0, f0);
    }
    {
        size_t f0 = J.size();
        dense(X(NL, 0), nullptr, T_(sTop), T[NL][0], nullptr, nullptr);
        step(P.trn, 0, f0);
    }
    for (int l = NL - 1; l >= 0; --l) {
        const int n = nl[l];
        if (l == 0) {
            size_t t0 = TJ.size();
            for (int i = 1, o = 0; i < n; i += 2, ++o)
                TJ.push_back(CRTriJob{Z[0][o], T[0][i], i + 1 < n ? X(0, i + 1) : nullptr, X(0, i - 1),
                                      i + 1 < n ? i + 1 : -1, i - 1});
            step(P.trn, 2, t0);
        } else {
            size_t f0 = J.size();
            for (int i = 1, o = 0; i < n; i += 2, ++o)
                dense(Z[l][o], T[l][i], i + 1 < n ? T_(sL[l][i + 1]) : nullptr, i + 1 < n ? X(l, i + 1) : nullptr,
                      T_(sU[l][i - 1]), X(l, i - 1));
            step(P.trn, 0, f0);
        }
        size_t f0 = J.size();
        for (int i = 1, o = 0; i < n; i += 2, ++o) dense(X(l, i), nullptr, T_(sDinv[l][o]), Z[l][o], nullptr, nullptr);
        step(P.trn, 0, f0);
    }
    for (const auto& j : J)
        if (!j.M1 || !j.v1 || !j.y) return fail(LS_ECUDA, "cyclic reduction: incomplete job table");
    CK(P.jobs.alloc(J.size()));
    CK(cudaMemcpy(P.jobs.p, J.data(), sizeof(CRJob) * J.size(), cudaMemcpyHostToDevice));
    P.hjobs = J;
    if (!TJ.empty()) {
        CK(P.tjobs.alloc(TJ.size()));
        CK(cudaMemcpy(P.tjobs.p, TJ.data(), sizeof(CRTriJob) * TJ.size(), cudaMemcpyHostToDevice));
    }
    return LS_OK;
}

// The steps of C x = t (transposed: C^T x = t) on P.t() -> P.x(), single right-hand side.
__global__ void k_to_dfc(int64_t n, const double2* __restrict__ a, float4* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 v = a[i];
    const float xh = (float)v.x, yh = (float)v.y;
    b[i] = make_float4(xh, yh, (float)(v.x - (double)xh), (float)(v.y - (double)yh));
}

// Double-float copy of the cyclic-reduction blocks and the job table pointing into it.
static ls_status ensure_cr_df(ls_op* op) {
    CRPlan& P = op->cr;
    if (P.store_df.p || P.hjobs.empty()) return LS_OK;
    const int64_t ns = (int64_t)P.store.n;
    CK(P.store_df.alloc(ns));
    k_to_dfc<<<(unsigned)((ns + 255) / 256), 256, 0, op->stream>>>(ns, P.store.p, P.store_df.p);
    CK(cudaGetLastError());
    op->launches++;
    std::vector<CRJobDF> JD(P.hjobs.size());
    for (size_t i = 0; i < JD.size(); ++i) {
        const CRJob& j = P.hjobs[i];
        const double2* m[2] = {j.M1, j.M2};
        const float4* md[2] = {nullptr, nullptr};
        for (int t = 0; t < 2; ++t) {
            if (!m[t]) continue;
            if (m[t] < P.store.p || m[t] >= P.store.p + ns) return fail(LS_ECUDA, "cyclic reduction: job outside the block store");
            md[t] = P.store_df.p + (m[t] - P.store.p);
        }
        JD[i] = CRJobDF{j.y, j.base, md[0], j.v1, md[1], j.v2};
    }
    CK(P.jobs_df.alloc(JD.size()));
    CK(cudaMemcpy(P.jobs_df.p, JD.data(), sizeof(CRJobDF) * JD.size(), cudaMemcpyHostToDevice));
    CK(raise_smem_limit(k_cr_mv_df, sizeof(float4) * 2 * P.nx));
    return LS_OK;
}

static int launch_cr(ls_op* op, cudaStream_t st, bool transposed, bool df = false) {
    const CRPlan& P = op->cr;
    const int nx = P.nx;
    const size_t shm = sizeof(double2) * 2 * nx;
    const int rows = CR_WARPS * CR_ROWS_PER_WARP;
    int nl = 0;
    for (const auto& s : transposed ? P.trn : P.fwd) {
        if (s.kind == 0 && df)
            k_cr_mv_df<<<dim3((nx + rows - 1) / rows, s.count, 1), 32 * CR_WARPS, sizeof(float4) * 2 * nx, st>>>(
                nx, P.jobs_df.p + s.first);
        else if (s.kind == 0)
            k_cr_mv<1><<<dim3((nx + rows - 1) / rows, s.count, 1), 32 * CR_WARPS, shm, st>>>(nx, 1, P.svec,
                                                                                         P.jobs.p + s.first);
        else
            k_cr_tri<<<dim3((nx + 127) / 128, s.count), 128, 0, st>>>(nx, 1, P.svec, op->cband.p, P.tjobs.p + s.first,
                                                                       s.kind == 2);
        ++nl;
    }
    return nl;
}

// The kernel sequence of P x on stream st (T_Q^C, the stencil A, the cyclic-reduction
// solve of C, then T_C^Q fused with the identity term); returns the number of launches.
static int launch_P_kernels(ls_op* op, cudaStream_t st, const double2* x, double2* z, bool df = false) {
    const int nc = op->nx * op->ny, nx = op->nx, ny = op->ny;
    k_tqc<<<(nc + 255) / 256, 256, 0, st>>>(nc, op->tqc_rp.p, op->tqc_ci.p, op->tqc_cv.p, x, op->pg.p);
    k_stencil<<<(nc + 255) / 256, 256, 0, st>>>(nx, ny, op->st.p, op->pg.p, op->cr.t());
    const int ncr = launch_cr(op, st, false, df);
    k_tcq<<<(op->nq + 255) / 256, 256, 0, st>>>(op->nq, op->tcq_idx.p, op->tcq_w.p, op->cr.x(), op->pg.p, x, z);
    return 3 + ncr;
}

// Cartesian operator: S^(C) x = C^{-1} A x; S^(C)^T x = A^T C^{-T} x.
static int launch_S_kernels(ls_op* op, cudaStream_t st, const double2* x, double2* z, bool transpose) {
    const int nc = op->nx * op->ny, nx = op->nx, ny = op->ny;
    if (!transpose) {
        k_stencil<<<(nc + 255) / 256, 256, 0, st>>>(nx, ny, op->st.p, x, op->cr.t());
        const int ncr = launch_cr(op, st, false);
        k_sub_vec<<<(nc + 255) / 256, 256, 0, st>>>(nc, op->cr.x(), op->czero.p, z);
        return 2 + ncr;
    }
    k_sub_vec<<<(nc + 255) / 256, 256, 0, st>>>(nc, x, op->czero.p, op->cr.t());
    const int ncr = launch_cr(op, st, true);
    k_stencilT<<<(nc + 255) / 256, 256, 0, st>>>(nx, ny, op->st.p, op->cr.x(), op->czero.p, z);
    return 2 + ncr;
}

// P^T x = x + T_Q^C^T (A^T C^{-T} - I) T_C^Q^T x on stream st; returns the number of launches.
static int launch_PT_kernels(ls_op* op, cudaStream_t st, const double2* x, double2* z, bool df = false) {
    const int nc = op->nx * op->ny, nx = op->nx, ny = op->ny;
    k_tqc<<<(nc + 255) / 256, 256, 0, st>>>(nc, op->tcqT_rp.p, op->tcqT_ci.p, op->tcqT_cv.p, x, op->cr.t());
    const int ncr = launch_cr(op, st, true, df);
    k_stencilT<<<(nc + 255) / 256, 256, 0, st>>>(nx, ny, op->st.p, op->cr.x(), op->cr.t(), op->ptp.p);
    k_tqcT<<<(op->nq + 255) / 256, 256, 0, st>>>(op->nq, op->tqcT_rp.p, op->tqcT_ci.p, op->tqcT_cv.p, op->ptp.p, nc, x,
                                                 op->nq, z, op->nq);
    return 3 + ncr;
}

// P x (transpose: P^T x).  Each sequence is captured once into a CUDA graph (on a
// private stream, with fixed input/output buffers) and replayed; x and z are copied
// in and out.
static ls_status apply_P_graph(ls_op* op, const double2* x, double2* z, bool transpose) {
    // the FP32 and mixed forms take the double-float blocks (their solves cannot see the
    // ~1e-13 rounding); the FP64-accurate forms keep the complex128 ones
    const bool df = !op->cartesian && (op->mode == 2 || op->mode == 4);
    if (df) TRY(ensure_cr_df(op));
    cudaGraphExec_t& ge = df ? (transpose ? op->gPTdf : op->gPdf) : (transpose ? op->gPT : op->gP);
    int& nlaunch = df ? (transpose ? op->nlaunch_PTdf : op->nlaunch_Pdf) : (transpose ? op->nlaunch_PT : op->nlaunch_P);
    if (!ge) {
        if (!op->cap) CK(cudaStreamCreateWithFlags(&op->cap, cudaStreamNonBlocking));
        if (!op->pin.p) CK(op->pin.alloc(op->nq));
        if (!op->pout.p) CK(op->pout.alloc(op->nq));
        CK(cudaStreamSynchronize(op->stream));           // the double-float blocks are ready before the capture
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(op->cap, cudaStreamCaptureModeThreadLocal));
        nlaunch = op->cartesian ? launch_S_kernels(op, op->cap, op->pin.p, op->pout.p, transpose)
                  : transpose   ? launch_PT_kernels(op, op->cap, op->pin.p, op->pout.p, df)
                                : launch_P_kernels(op, op->cap, op->pin.p, op->pout.p, df);
        CK(cudaStreamEndCapture(op->cap, &g));
        cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        CK(e);
    }
    CK(cudaMemcpyAsync(op->pin.p, x, sizeof(double2) * op->nq, cudaMemcpyDeviceToDevice, op->stream));
    CK(cudaGraphLaunch(ge, op->stream));
    CK(cudaMemcpyAsync(z, op->pout.p, sizeof(double2) * op->nq, cudaMemcpyDeviceToDevice, op->stream));
    op->launches += nlaunch;
    return LS_OK;
}

static ls_status apply_P(ls_op* op, const double2* x, double2* z) { return apply_P_graph(op, x, z, false); }

// y = L^T x (mode 0) or y = V^T x (mode 2)
static ls_status apply_LT(ls_op* op, const double2* x, double2* y, int mode = 0) {
    if (op->cartesian) return cart_apply(op, x, y, mode == 2 ? 2 : 1);   // V^(C) is symmetric
    ls_status s = launch_pairsum(op, x, nullptr, nullptr);
    if (s != LS_OK) return s;
    TRY(collapse_slots(op));
    int threads = 256;
    int blocks = (int)(((int64_t)op->nq * 32 + threads - 1) / threads);
    k_applyT_epi<<<blocks, threads, 0, op->stream>>>(op->nq, op->ps_slots, op->partial.p, op->rowptrT.p, op->colsT.p,
                                                     op->valsT.p, op->m.p, op->w.p, x, op->k * op->k, y, mode);
    CK(cudaGetLastError());
    op->launches++;
    return LS_OK;
}

// z = P^T x = x + T_Q^C^T (A^T C^{-T} - I) T_C^Q^T x
static ls_status apply_PT(ls_op* op, const double2* x, double2* z) { return apply_P_graph(op, x, z, true); }

// h[0:J] = V[0:J]^H z (into dst, accumulate or overwrite)
static ls_status dots(ls_op* op, int J, const double2* V, const double2* z, double2* dst, int accumulate) {
    k_dots<<<op->dblk, RED_TPB, 0, op->stream>>>(op->nq, J, V, (size_t)op->nq, z, op->dpart.p);
    k_sumrows<<<(J + 127) / 128, 128, 0, op->stream>>>(J, op->dblk, op->dpart.p, dst, accumulate);
    CK(cudaGetLastError());
    op->launches += 2;
    return LS_OK;
}


// One GMRES solve for device rhs b -> u. Writes hist (host, may be null) and iterations.
static ls_status gmres_one(ls_op* op, const double2* b, double2* u, double* hist_host, int* iters, bool transpose = false) {
    auto opL = [&](const double2* x, double2* y) { return transpose ? apply_LT(op, x, y) : apply_L(op, x, y); };
    auto opP = [&](const double2* x, double2* y) { return transpose ? apply_PT(op, x, y) : apply_P(op, x, y); };
    const int n = op->nq, maxit = op->prm.max_iter;
    const int ldh = maxit + 1;
    const size_t ldv = (size_t)n;
    const int tpb = 256, nb = (n + tpb - 1) / tpb;
    double2* V = op->Vb.p;
    CK(cudaMemsetAsync(op->H.p, 0, sizeof(double2) * (size_t)ldh * maxit, op->stream));
    // r0 = P b
    if (op->has_prec && op->prm.use_precond) TRY(opP(b, op->tmp.p));
    else CK(cudaMemcpyAsync(op->tmp.p, b, sizeof(double2) * n, cudaMemcpyDeviceToDevice, op->stream));
    TRY(dots(op, 1, op->tmp.p, op->tmp.p, op->scal.p, 0));       // scal[0] = ||r0||^2
    k_scale<<<nb, tpb, 0, op->stream>>>(n, op->tmp.p, op->scal.p, V, nullptr);
    k_gmres_init<<<1, 1, 0, op->stream>>>(op->g.p, op->scal.p, op->hist.p);
    CK(cudaGetLastError());
    op->launches += 2;
    int it = 0;
    bool conv = false;
    double last = 1.0;
    for (int j = 0; j < maxit; ++j) {
        double2* vj = V + (size_t)j * ldv;
        double2* vn = V + (size_t)(j + 1) * ldv;
        double2* hcol = op->H.p + (size_t)j * ldh;
        if (op->has_prec && op->prm.use_precond) {
            TRY(opL(vj, op->tmp.p));
            TRY(opP(op->tmp.p, vn));
        } else {
            TRY(opL(vj, vn));
        }
        CK(cudaMemcpyAsync(op->Wb.p + (size_t)j * ldv, vn, sizeof(double2) * n, cudaMemcpyDeviceToDevice, op->stream));
        // classical Gram-Schmidt, twice
        TRY(dots(op, j + 1, V, vn, hcol, 0));
        k_update<<<nb, tpb, sizeof(double2) * (j + 1), op->stream>>>(n, j + 1, V, ldv, hcol, vn);
        TRY(dots(op, j + 1, V, vn, op->hv.p, 0));
        k_update<<<nb, tpb, sizeof(double2) * (j + 1), op->stream>>>(n, j + 1, V, ldv, op->hv.p, vn);
        k_sumrows<<<(j + 1 + 127) / 128, 128, 0, op->stream>>>(j + 1, 1, op->hv.p, hcol, 1);
        TRY(dots(op, 1, vn, vn, op->scal.p + 1, 0));
        k_scale<<<nb, tpb, 0, op->stream>>>(n, vn, op->scal.p + 1, vn, hcol + j + 1);
        CK(cudaMemcpyAsync(op->Hraw.p + (size_t)j * ldh, hcol, sizeof(double2) * (j + 2), cudaMemcpyDeviceToDevice,
                           op->stream));
        k_givens<<<1, 1, 0, op->stream>>>(j, op->H.p, ldh, op->cs.p, op->sn.p, op->g.p, op->hist.p, op->scal.p);
        CK(cudaGetLastError());
        op->launches += 5;
        CK(cudaMemcpyAsync(&last, op->hist.p + j + 1, sizeof(double), cudaMemcpyDeviceToHost, op->stream));
        CK(cudaStreamSynchronize(op->stream));
        it = j + 1;
        if (!(last > op->prm.tol)) { conv = true; break; }
    }
    k_backsolve<<<1, 1, 0, op->stream>>>(it, op->H.p, ldh, op->g.p, op->yv.p);
    k_combine<<<nb, tpb, sizeof(double2) * it, op->stream>>>(n, it, V, ldv, op->yv.p, u);
    // explicit residual at exit: P b - sum_i y_i (P L v_i) from the stored operator products
    // (it does not rely on the orthogonality of the basis the Givens estimate assumes)
    k_combine<<<nb, tpb, sizeof(double2) * it, op->stream>>>(n, it, op->Wb.p, ldv, op->yv.p, op->tmp2.p);
    k_resid_check<<<nb, tpb, 0, op->stream>>>(n, V, op->scal.p, op->tmp2.p, op->tmp.p);
    CK(cudaGetLastError());
    op->launches += 4;
    TRY(dots(op, 1, op->tmp.p, op->tmp.p, op->scal.p + 2, 0));
    double2 sc[3];
    CK(cudaMemcpyAsync(sc, op->scal.p, sizeof(double2) * 3, cudaMemcpyDeviceToHost, op->stream));
    if (hist_host) CK(cudaMemcpyAsync(hist_host, op->hist.p, sizeof(double) * (it + 1), cudaMemcpyDeviceToHost, op->stream));
    CK(cudaStreamSynchronize(op->stream));
    const double rel = sc[0].x > 0 ? std::sqrt(sc[2].x / sc[0].x) : 0.0;
    op->last_res = std::max(op->last_res, rel);
    op->last_it = it;
    if (iters) *iters = it;
    if (conv && !(rel <= 10.0 * op->prm.tol)) {
        fail(LS_ENOCONV, "GMRES: explicit residual " + std::to_string(rel) + " exceeds 10 x tol");
        return LS_ENOCONV;
    }
    return conv ? LS_OK : LS_ENOCONV;
}

// ||P (b - L u)|| / ||P b|| by full applies of L and P (||b - L u|| / ||b|| without P).
static ls_status residual_full(ls_op* op, const double2* b, const double2* u, double* rel) {
    const int n = op->nq, nb = (n + 255) / 256;
    DevBuf<double2> r, pr, pb;
    CK(r.alloc(n));
    CK(pr.alloc(n));
    CK(pb.alloc(n));
    TRY(apply_L(op, u, op->tmp2.p));
    k_sub_vec<<<nb, 256, 0, op->stream>>>(n, b, op->tmp2.p, r.p);
    CK(cudaGetLastError());
    const bool prec = op->has_prec && op->prm.use_precond;
    if (prec) {
        TRY(apply_P(op, r.p, pr.p));
        TRY(apply_P(op, b, pb.p));
    } else {
        CK(cudaMemcpyAsync(pr.p, r.p, sizeof(double2) * n, cudaMemcpyDeviceToDevice, op->stream));
        CK(cudaMemcpyAsync(pb.p, b, sizeof(double2) * n, cudaMemcpyDeviceToDevice, op->stream));
    }
    TRY(dots(op, 1, pr.p, pr.p, op->scal.p + 2, 0));
    TRY(dots(op, 1, pb.p, pb.p, op->scal.p + 3, 0));
    double2 sc[2];
    CK(cudaMemcpyAsync(sc, op->scal.p + 2, sizeof(double2) * 2, cudaMemcpyDeviceToHost, op->stream));
    CK(cudaStreamSynchronize(op->stream));
    *rel = sc[1].x > 0 ? std::sqrt(sc[0].x / sc[1].x) : 0.0;
    return LS_OK;
}

// Mixed-precision solve (pairsum mode 4): GMRES with the FP32 pair sum, then iterative
// refinement against the double-float (FP64-accurate) operator.  The residual of the FP32
// solution, r = b - L u, is formed with the accurate L; while ||P r|| > tol ||P b|| an FP32
// GMRES solves L d = r to the relative tolerance that brings ||P r|| below tol / 2 (at most
// 0.5, at least 1e-3, where the FP32 operator's own error starts to limit the correction),
// u += d and r -= L d (FP32: the product of the small correction needs no more).  The
// exit residual (ls_op_last_residual) is that residual's.
#define MIXED_REFINE 4
static ls_status solve_mixed(ls_op* op, const double2* b, double2* u, double* hist_host, int* iters, bool transpose) {
    const int n = op->nq, nb = (n + 255) / 256;
    const double tol = op->prm.tol;
    const double lr0 = op->last_res;
    const bool prec = op->has_prec && op->prm.use_precond;
    if (op->ir_r.n < (size_t)n) {
        CK(op->ir_r.alloc(n));
        CK(op->ir_d.alloc(n));
        CK(op->ir_y.alloc(n));
    }
    op->inner32 = true;
    int it = 0;
    ls_status s = gmres_one(op, b, u, hist_host, &it, transpose);
    op->inner32 = false;
    if (s != LS_OK && s != LS_ENOCONV) return s;
    int total = it;
    // ||P x||^2 into scal[slot] (ir_y as scratch)
    auto pnorm2 = [&](const double2* x, int slot, double& out) -> ls_status {
        const double2* px = x;
        if (prec) {
            TRY(transpose ? apply_PT(op, x, op->ir_y.p) : apply_P(op, x, op->ir_y.p));
            px = op->ir_y.p;
        }
        TRY(dots(op, 1, px, px, op->scal.p + slot, 0));
        double2 v;
        CK(cudaMemcpyAsync(&v, op->scal.p + slot, sizeof(double2), cudaMemcpyDeviceToHost, op->stream));
        CK(cudaStreamSynchronize(op->stream));
        out = v.x;
        return LS_OK;
    };
    double pb2 = 0, pr2 = 0, rel = 0;
    TRY(pnorm2(b, 3, pb2));
    for (int step = 0;; ++step) {
        if (step == 0) {
            // r = b - L u with the double-float operator
            TRY(transpose ? apply_LT(op, u, op->ir_y.p) : apply_L(op, u, op->ir_y.p));
            k_sub_vec<<<nb, 256, 0, op->stream>>>(n, b, op->ir_y.p, op->ir_r.p);
        } else {
            // after u += d: r -= L d with the FP32 operator.  Its error is relative to |d|,
            // eps32 ||k^2 V M|| ||d|| <= eps32 cond(L) ||r||, about 1e-13 of ||b|| for an FP32
            // solve's residual of ~1e-7 ||b||: far below tol
            op->inner32 = true;
            ls_status sa = transpose ? apply_LT(op, op->ir_d.p, op->ir_y.p) : apply_L(op, op->ir_d.p, op->ir_y.p);
            op->inner32 = false;
            TRY(sa);
            k_sub_vec<<<nb, 256, 0, op->stream>>>(n, op->ir_r.p, op->ir_y.p, op->ir_r.p);
        }
        CK(cudaGetLastError());
        op->launches++;
        TRY(pnorm2(op->ir_r.p, 2, pr2));
        rel = pb2 > 0 ? std::sqrt(pr2 / pb2) : 0.0;
        if (rel <= tol || step == MIXED_REFINE) break;
        const double tol_save = op->prm.tol;
        op->prm.tol = std::min(0.5, std::max(0.5 * tol / rel, 1e-3));
        op->inner32 = true;
        ls_status sc = gmres_one(op, op->ir_r.p, op->ir_d.p, nullptr, &it, transpose);
        op->inner32 = false;
        op->prm.tol = tol_save;
        if (sc != LS_OK && sc != LS_ENOCONV) return sc;
        total += it;
        k_accumulate_multi<<<nb, 256, 0, op->stream>>>(n, op->ir_d.p, u);
        CK(cudaGetLastError());
        op->launches++;
    }
    op->last_res = std::max(lr0, rel);
    op->last_it = total;
    if (iters) *iters = total;
    if (rel <= tol) return LS_OK;
    fail(LS_ENOCONV, "mixed-precision refinement: residual " + std::to_string(rel) + " above tol");
    return LS_ENOCONV;
}

// One single-RHS solve in the operator's pair-sum form.
static ls_status solve_one(ls_op* op, const double2* b, double2* u, double* hist_host, int* iters,
                           bool transpose = false) {
    if (op->mode == 4 && !op->cartesian) return solve_mixed(op, b, u, hist_host, iters, transpose);
    return gmres_one(op, b, u, hist_host, iters, transpose);
}

// Error reporting for other translation units of the library.
ls_status lsgpu_set_error(ls_status s, const char* msg) { return fail(s, msg); }

// ------------------------------------------------------------------ C ABI
extern "C" {

const char* ls_last_error(void) { return g_err.c_str(); }

void ls_params_default(ls_params* p) {
    if (!p) return;
    p->tol = 1e-8;
    p->max_iter = 600;
    p->use_precond = 1;
    p->kappa = 3.0;
    p->box[0] = -1.2; p->box[1] = 1.2; p->box[2] = -1.2; p->box[3] = 1.2;
    p->nx = 256;
    p->ny = 256;
    p->prec = LS_PREC_FP64_DF;
    p->approach = 2;
    p->setup_on_device = 1;
}

ls_status ls_mesh_create(int32_t n_vert, const double* vert_xy, int32_t n_elem, const int32_t* elem_vert,
                         const int32_t* elem_domain, const int32_t* edge_curve, const double* edge_theta,
                         int32_t n_curve, const double* curves, const double* nodes_xy, const double* weights,
                         ls_mesh** out) {
    if (!out) return fail(LS_EINVAL, "out is null");
    *out = nullptr;
    if (n_vert < 3 || n_elem < 1 || !vert_xy || !elem_vert || !elem_domain || !edge_curve || !edge_theta ||
        !nodes_xy || !weights || n_curve < 0 || (n_curve > 0 && !curves))
        return fail(LS_EINVAL, "ls_mesh_create: null pointer or bad size");
    ls_mesh* M = new (std::nothrow) ls_mesh;
    if (!M) return fail(LS_ENOMEM, "host allocation");
    HostMesh& h = M->h;
    h.nv = n_vert; h.nt = n_elem; h.nq = n_elem * lsgpu::NQ_ELEM; h.ncurve = n_curve;
    h.vxy.assign(vert_xy, vert_xy + 2 * (size_t)n_vert);
    h.tri.assign(elem_vert, elem_vert + 3 * (size_t)n_elem);
    h.dom.assign(elem_domain, elem_domain + n_elem);
    h.ecurve.assign(edge_curve, edge_curve + 3 * (size_t)n_elem);
    h.etheta.assign(edge_theta, edge_theta + 6 * (size_t)n_elem);
    h.curves.assign(curves, curves + 6 * (size_t)n_curve);
    h.nodes.assign(nodes_xy, nodes_xy + 2 * (size_t)h.nq);
    h.w.assign(weights, weights + h.nq);
    for (int t = 0; t < n_elem; ++t) {
        for (int e = 0; e < 3; ++e) {
            int v = h.tri[3 * t + e];
            int c = h.ecurve[3 * t + e];
            if (v < 0 || v >= n_vert || c < -1 || c >= n_curve) { delete M; return fail(LS_EINVAL, "element index out of range"); }
        }
        if (h.dom[t] < 0) { delete M; return fail(LS_EINVAL, "negative subdomain id"); }
        const int* v = &h.tri[3 * t];
        double ax = h.vxy[2 * v[1]] - h.vxy[2 * v[0]], ay = h.vxy[2 * v[1] + 1] - h.vxy[2 * v[0] + 1];
        double bx = h.vxy[2 * v[2]] - h.vxy[2 * v[0]], by = h.vxy[2 * v[2] + 1] - h.vxy[2 * v[0] + 1];
        if (!(ax * by - ay * bx > 0)) { delete M; return fail(LS_EINVAL, "clockwise or degenerate element " + std::to_string(t)); }
    }
    for (int q = 0; q < h.nq; ++q)
        if (!std::isfinite(h.nodes[2 * q]) || !std::isfinite(h.nodes[2 * q + 1]) || !std::isfinite(h.w[q])) {
            delete M;
            return fail(LS_EINVAL, "non-finite node or weight");
        }
    *out = M;
    return LS_OK;
}

void ls_mesh_destroy(ls_mesh* mesh) { delete mesh; }
int32_t ls_mesh_num_nodes(const ls_mesh* mesh) { return mesh ? mesh->h.nq : 0; }
int32_t ls_op_num_nodes(const ls_op* op) { return op ? op->nq : 0; }

// Tabulated H0 for the pair sum: t from (1e-2 h_min)^2 to the squared bounding-box diagonal.
static ls_status build_table_range(ls_op* op, double t_lo, double t_hi, int mode);

// FP32 table layout: coef [ncell][NC_F32] float2, cells (mid_hi, mid_lo, inv_hw, 0), oct (base, 23 - m)
static ls_status upload_f32_table(const lsgpu::H0Table& T, DevBuf<double2>& buf, int& ncell, int& noct, int& blo,
                                  size_t& bytes, double& err) {
    ncell = (int)T.mid.size();
    const int coef_f4 = (ncell * NC_F32 + 1) / 2;
    std::vector<float4> hf((size_t)coef_f4 + ncell + (T.noct + 1) / 2, make_float4(0.f, 0.f, 0.f, 0.f));
    float2* cf = reinterpret_cast<float2*>(hf.data());
    for (size_t i = 0; i < (size_t)ncell * NC_F32; ++i) cf[i] = make_float2((float)T.coef[i].real(), (float)T.coef[i].imag());
    for (int c = 0; c < ncell; ++c) {
        float mh = (float)T.mid[c];
        hf[(size_t)coef_f4 + c] = make_float4(mh, (float)(T.mid[c] - (double)mh), (float)T.inv_hw[c], 0.f);
    }
    int2* oct = reinterpret_cast<int2*>(hf.data() + coef_f4 + ncell);
    for (int o = 0; o < T.noct; ++o) oct[o] = make_int2(T.oct_base[o], T.oct_shift[o] + 3);
    noct = T.noct;
    blo = T.b_lo - 1023 + 127;
    err = T.max_rel_err;
    bytes = hf.size() * sizeof(float4);
    CK(buf.alloc((bytes + sizeof(double2) - 1) / sizeof(double2)));
    CK(cudaMemcpy(buf.p, hf.data(), bytes, cudaMemcpyHostToDevice));
    return LS_OK;
}

static ls_status ensure_table32(ls_op* op) {
    if (op->t32_bytes) return LS_OK;
    lsgpu::H0Table T;
    std::string err = lsgpu::build_h0_table(op->k, op->tab_tlo, op->tab_thi, T, NC_F32, 2e-8);
    if (!err.empty()) return fail(LS_EINVAL, err);
    double e = 0;
    TRY(upload_f32_table(T, op->tab32, op->t32_ncell, op->t32_noct, op->t32_blo, op->t32_bytes, e));
    CK(raise_smem_limit(k_pairsum_multi_f32, op->t32_bytes));
    return LS_OK;
}

// The FP32 table of the mixed form's inner solves (shared with the batched kernels).
static ls_status ensure_table32_single(ls_op* op) {
    TRY(ensure_table32(op));
    CK(raise_smem_limit(k_pairsum_f32, op->t32_bytes));
    CK(raise_smem_limit(k_pairsum_f32s, op->t32_bytes));
    return LS_OK;
}

static void table_range(ls_op* op, const HostMesh& M) {
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300, hmin = 1e300;
    for (int q = 0; q < M.nq; ++q) {
        xmin = std::min(xmin, M.nodes[2 * q]); xmax = std::max(xmax, M.nodes[2 * q]);
        ymin = std::min(ymin, M.nodes[2 * q + 1]); ymax = std::max(ymax, M.nodes[2 * q + 1]);
    }
    for (int t = 0; t < M.nt; ++t) {
        const int* v = &M.tri[3 * t];
        for (int e = 0; e < 3; ++e) {
            double dx = M.vxy[2 * v[e]] - M.vxy[2 * v[(e + 1) % 3]], dy = M.vxy[2 * v[e] + 1] - M.vxy[2 * v[(e + 1) % 3] + 1];
            hmin = std::min(hmin, std::sqrt(dx * dx + dy * dy));
        }
    }
    double t_hi = ((xmax - xmin) * (xmax - xmin) + (ymax - ymin) * (ymax - ymin)) * 1.0001;
    double t_lo = std::min(1e-2 * hmin * 1e-2 * hmin, t_hi / 4);
    op->tab_tlo = t_lo;
    op->tab_thi = t_hi;
}

// Upload an FP64 (mode 0) or double-float (mode 3) table with nc coefficients per cell.
static ls_status upload_table(ls_op* op, const lsgpu::H0Table& T, int nc, int mode) {
    const int ncell = (int)T.mid.size();
    if (mode == 3) {
        std::vector<float4> hd((size_t)ncell * (nc + 1) + (T.noct + 1) / 2, make_float4(0.f, 0.f, 0.f, 0.f));
        auto split = [](double x, float& h, float& l) { h = (float)x; l = (float)(x - (double)h); };
        for (size_t i = 0; i < (size_t)ncell * nc; ++i) {
            float a, b, c, d;
            split(T.coef[i].real(), a, b);
            split(T.coef[i].imag(), c, d);
            hd[i] = make_float4(a, b, c, d);
        }
        for (int c = 0; c < ncell; ++c) {
            float a, b;
            split(T.mid[c], a, b);
            hd[(size_t)ncell * nc + c] = make_float4(a, b, (float)T.inv_hw[c], 0.f);
        }
        int2* oct = reinterpret_cast<int2*>(hd.data() + (size_t)ncell * (nc + 1));
        for (int o = 0; o < T.noct; ++o) oct[o] = make_int2(T.oct_base[o], T.oct_shift[o] + 3);
        op->tab_blo = T.b_lo - 1023 + 127;
        // FP32 tail: the top nf coefficients may be summed in FP32 when, on every cell, their
        // total magnitude (|u| <= 1) times nf 2^-24 stays below 2^-50 of |H0| on the cell (its
        // smallest value at 17 equispaced samples; H0 has no zero on a cell of the table range)
        op->tab_nf = 0;
        for (int nf : {4, 2}) {
            if (nf >= nc - 2) continue;
            bool ok = true;
            for (int c = 0; c < ncell && ok; ++c) {
                const std::complex<double>* cc = &T.coef[(size_t)c * nc];
                double tail = 0;
                for (int e = nc - nf; e < nc; ++e) tail += std::abs(cc[e]);
                double hmin = 1e300;
                for (int q = 0; q <= 16; ++q) {
                    const double u = -1.0 + q / 8.0;
                    std::complex<double> p = 0;
                    for (int e = nc - 1; e >= 0; --e) p = p * u + cc[e];
                    hmin = std::min(hmin, std::abs(p));
                }
                ok = tail * nf * std::ldexp(1.0, -24) <= std::ldexp(1.0, -50) * hmin;
            }
            if (ok) { op->tab_nf = nf; break; }
        }
        op->tab_bytes = hd.size() * sizeof(float4);
        CK(op->tab.alloc((op->tab_bytes + sizeof(double2) - 1) / sizeof(double2)));
        CK(cudaMemcpy(op->tab.p, hd.data(), op->tab_bytes, cudaMemcpyHostToDevice));
    } else {
        std::vector<double2> h((size_t)ncell * (nc + 1) + (T.noct + 1) / 2);
        for (size_t i = 0; i < (size_t)ncell * nc; ++i) h[i] = make_double2(T.coef[i].real(), T.coef[i].imag());
        for (int c = 0; c < ncell; ++c) h[(size_t)ncell * nc + c] = make_double2(T.mid[c], T.inv_hw[c]);
        int2* oct = reinterpret_cast<int2*>(h.data() + (size_t)ncell * (nc + 1));
        for (int o = 0; o < T.noct; ++o) oct[o] = make_int2(T.oct_base[o], T.oct_shift[o]);
        op->tab_blo = T.b_lo;
        op->tab_bytes = h.size() * sizeof(double2);
        CK(op->tab.alloc(h.size()));
        CK(cudaMemcpy(op->tab.p, h.data(), op->tab_bytes, cudaMemcpyHostToDevice));
    }
    op->tab_ncell = ncell;
    op->tab_noct = T.noct;
    op->tab_err = T.max_rel_err;
    op->tab_nc = nc;
    CK(raise_tab_limits(mode, op->tab_bytes));
    return LS_OK;
}

// Tables for the pair sum.  Modes 0 and 3 autotune the polynomial degree: every
// candidate (12, 10 or 9 coefficients per cell, each validated to 2e-15 at build
// time, with fewer cells for higher degree) whose table fits in shared memory is
// timed on one pair-sum launch over the operator's own nodes; the fastest is kept.
static ls_status build_table_range(ls_op* op, double t_lo, double t_hi, int mode) {
    if (mode == 2) {
        lsgpu::H0Table T;
        std::string err = lsgpu::build_h0_table(op->k, t_lo, t_hi, T, NC_F32, 2e-8);
        if (!err.empty()) return fail(LS_EINVAL, err);
        double err32 = 0;
        TRY(upload_f32_table(T, op->tab, op->tab_ncell, op->tab_noct, op->tab_blo, op->tab_bytes, err32));
        op->tab_err = err32;
        CK(raise_smem_limit(k_pairsum_f32, op->tab_bytes));
        CK(raise_smem_limit(k_pairsum_f32s, op->tab_bytes));
        op->use_table = true;
        return LS_OK;
    }
    const int cand[4] = {12, 10, 9, 8};
    const int ncand = mode == 3 ? 4 : 3;
    const size_t smem_cap = 160 * 1024;
    DevBuf<double2> fdum;
    CK(fdum.alloc(op->nq));
    CK(cudaMemsetAsync(fdum.p, 0, sizeof(double2) * op->nq, op->stream));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int best_nc = 12;
    float best = 1e30f;
    dim3 grid((op->nq + PS_TPB - 1) / PS_TPB, op->nchunk);
    // time each candidate on at most ~2e9 pairs: the first spc_t sources of every chunk
    // (same per-pair work and launch shape; the time is scaled to the full launch)
    const double pairs_cap = 2e9;
    int spc_t = op->src_per_chunk;
    if ((double)op->nq * op->nq > pairs_cap) {
        spc_t = (int)std::ceil(pairs_cap / ((double)op->nq * op->nchunk));
        spc_t = std::min(op->src_per_chunk, ((spc_t + PS_TILE - 1) / PS_TILE) * PS_TILE);
    }
    const int n_t = op->nchunk > 1 ? op->nq : std::min(op->nq, spc_t);   // one chunk: stop at spc_t sources
    const float scale_t = (float)op->src_per_chunk / (float)spc_t;
    for (int c = 0; c < ncand; ++c) {
        lsgpu::H0Table T;
        std::string err = lsgpu::build_h0_table(op->k, t_lo, t_hi, T, cand[c], 2e-15);
        op->tune_ms[c] = 0.f;
        if (!err.empty() || T.max_rel_err > 2e-15) continue;
        size_t words = T.mid.size() * (cand[c] + 1) + (T.noct + 1) / 2;
        if (words * 16 > smem_cap) continue;
        TRY(upload_table(op, T, cand[c], mode));
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {          // first launch warms up, second is timed
            CK(cudaEventRecord(e0, op->stream));
            if (mode == 3)
                launch_df(cand[c], op->tab_nf, grid, op->tab_bytes, op->stream, op->xy.p, op->w.p, nullptr, fdum.p, n_t,
                          spc_t, op->k, (const float4*)op->tab.p, op->tab_ncell, op->tab_noct, op->tab_blo,
                          op->partial.p);
            else
                launch_tab(cand[c], grid, op->tab_bytes, op->stream, op->xy.p, op->w.p, nullptr, fdum.p, n_t,
                           spc_t, op->k, op->tab.p, op->tab_ncell, op->tab_noct, op->tab_blo, op->partial.p);
            CK(cudaGetLastError());
            CK(cudaEventRecord(e1, op->stream));
            CK(cudaEventSynchronize(e1));
            CK(cudaEventElapsedTime(&ms, e0, e1));
        }
        ms *= scale_t;
        op->tune_ms[c] = ms;
        if (ms < best) { best = ms; best_nc = cand[c]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    lsgpu::H0Table T;
    std::string err = lsgpu::build_h0_table(op->k, t_lo, t_hi, T, best_nc, 2e-15);
    if (!err.empty()) return fail(LS_EINVAL, err);
    TRY(upload_table(op, T, best_nc, mode));
    op->use_table = true;
    return LS_OK;
}
static ls_status build_preconditioner(ls_op* op, const HostMesh& M, const double* m_grid) {
    GridSetup G;
    std::vector<std::complex<double>> mg((size_t)op->prm.nx * op->prm.ny);
    for (size_t i = 0; i < mg.size(); ++i) {
        mg[i] = std::complex<double>(m_grid[2 * i], m_grid[2 * i + 1]);
        if (!std::isfinite(mg[i].real()) || !std::isfinite(mg[i].imag())) return fail(LS_EINVAL, "non-finite m_grid");
    }
    auto tg0 = std::chrono::steady_clock::now();
    std::string err = lsgpu::build_grid(M, op->k, op->prm.box, op->prm.nx, op->prm.ny, mg.data(), G, op->prm.approach);
    if (!err.empty()) return fail(LS_EINVAL, err);
    op->t_setup[1] = std::chrono::duration<double>(std::chrono::steady_clock::now() - tg0).count();
    auto tl0 = std::chrono::steady_clock::now();
    const int nx = G.nx, ny = G.ny, nc = nx * ny;
    op->nx = nx; op->ny = ny;
    {
        std::vector<double2> hs(81);
        for (int c = 0; c < 9; ++c)
            for (int t = 0; t < 9; ++t) hs[9 * c + t] = make_double2(G.v[c][t].real(), G.v[c][t].imag());
        CK(op->st.alloc(81));
        CK(cudaMemcpy(op->st.p, hs.data(), sizeof(double2) * 81, cudaMemcpyHostToDevice));
    }
    CK(op->tcq_idx.alloc(G.tcq_idx.size()));
    CK(op->tcq_w.alloc(G.tcq_w.size()));
    CK(op->tqc_rp.alloc(G.tqc_rowptr.size()));
    CK(op->tqc_ci.alloc(G.tqc_cols.size()));
    CK(op->tqc_cv.alloc(G.tqc_vals.size()));
    CK(op->cband.alloc(G.cband.size()));
    CK(cudaMemcpy(op->tcq_idx.p, G.tcq_idx.data(), sizeof(int) * G.tcq_idx.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->tcq_w.p, G.tcq_w.data(), sizeof(double) * G.tcq_w.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->tqc_rp.p, G.tqc_rowptr.data(), sizeof(int64_t) * G.tqc_rowptr.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->tqc_ci.p, G.tqc_cols.data(), sizeof(int) * G.tqc_cols.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->tqc_cv.p, G.tqc_vals.data(), sizeof(double) * G.tqc_vals.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->cband.p, G.cband.data(), sizeof(double2) * G.cband.size(), cudaMemcpyHostToDevice));
    CK(op->tcqT_rp.alloc(G.tcqT_rowptr.size()));
    CK(op->tcqT_ci.alloc(G.tcqT_cols.size()));
    CK(op->tcqT_cv.alloc(G.tcqT_vals.size()));
    CK(op->tqcT_rp.alloc(G.tqcT_rowptr.size()));
    CK(op->tqcT_ci.alloc(std::max<size_t>(1, G.tqcT_cols.size())));
    CK(op->tqcT_cv.alloc(std::max<size_t>(1, G.tqcT_vals.size())));
    CK(cudaMemcpy(op->tcqT_rp.p, G.tcqT_rowptr.data(), sizeof(int64_t) * G.tcqT_rowptr.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->tcqT_ci.p, G.tcqT_cols.data(), sizeof(int) * G.tcqT_cols.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->tcqT_cv.p, G.tcqT_vals.data(), sizeof(double) * G.tcqT_vals.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->tqcT_rp.p, G.tqcT_rowptr.data(), sizeof(int64_t) * G.tqcT_rowptr.size(), cudaMemcpyHostToDevice));
    if (!G.tqcT_cols.empty()) {
        CK(cudaMemcpy(op->tqcT_ci.p, G.tqcT_cols.data(), sizeof(int) * G.tqcT_cols.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(op->tqcT_cv.p, G.tqcT_vals.data(), sizeof(double) * G.tqcT_vals.size(), cudaMemcpyHostToDevice));
    }
    op->n_interior = G.n_interior;
    CK(op->Dg.alloc(nc));
    CK(cudaMemcpy(op->Dg.p, G.D.data(), sizeof(double) * nc, cudaMemcpyHostToDevice));
    CK(op->pg.alloc(nc));
    CK(op->pt.alloc(nc));
    CK(op->ptp.alloc(nc));
    CK(op->Wf.alloc((size_t)ny * nx * nx));
    CK(op->Gf.alloc((size_t)ny * nx * nx));
    // block LU: S_b = C_bb - C_{b,b-1} G_{b-1}; W_b = S_b^{-1}; G_b = W_b C_{b,b+1}
    cusolverDnHandle_t hs = nullptr;
    CKS(cusolverDnCreate(&hs));
    struct HG { cusolverDnHandle_t h; ~HG() { cusolverDnDestroy(h); } } guard{hs};
    CKS(cusolverDnSetStream(hs, op->stream));
    DevBuf<double2> S, X, work;
    DevBuf<int> piv, info;
    CK(S.alloc((size_t)nx * nx));
    CK(X.alloc((size_t)nx * nx));
    CK(piv.alloc(nx));
    CK(info.alloc(1));
    int lwork = 0;
    CKS(cusolverDnZgetrf_bufferSize(hs, nx, nx, (cuDoubleComplex*)S.p, nx, &lwork));
    CK(work.alloc(std::max(lwork, 1)));
    dim3 blk(128), grd((nx + 127) / 128, nx);
    for (int b = 0; b < ny; ++b) {
        k_build_S<<<grd, blk, 0, op->stream>>>(nx, b, op->cband.p, b > 0 ? op->Gf.p + (size_t)(b - 1) * nx * nx : nullptr, S.p);
        CK(cudaGetLastError());
        CKS(cusolverDnZgetrf(hs, nx, nx, (cuDoubleComplex*)S.p, nx, (cuDoubleComplex*)work.p, piv.p, info.p));
        int hinfo = 0;
        CK(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, op->stream));
        CK(cudaStreamSynchronize(op->stream));
        if (hinfo != 0) return fail(LS_ESINGULAR, "block " + std::to_string(b) + " of C is singular");
        k_identity_cm<<<grd, blk, 0, op->stream>>>(nx, X.p);
        CKS(cusolverDnZgetrs(hs, CUBLAS_OP_N, nx, nx, (const cuDoubleComplex*)S.p, nx, piv.p, (cuDoubleComplex*)X.p, nx, info.p));
        k_store_W_G<<<grd, blk, 0, op->stream>>>(nx, b, ny, X.p, op->cband.p, op->Wf.p, op->Gf.p);
        CK(cudaGetLastError());
    }
    CK(op->WT.alloc((size_t)ny * nx * nx));
    CK(op->GT.alloc((size_t)ny * nx * nx));
    {
        dim3 tb(32, 8), tg((nx + 31) / 32, (nx + 31) / 32, ny);
        k_transpose_blocks<<<tg, tb, 0, op->stream>>>(nx, ny, op->Wf.p, op->WT.p);
        k_transpose_blocks<<<tg, tb, 0, op->stream>>>(nx, ny, op->Gf.p, op->GT.p);
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(op->stream));
    TRY(build_cr(op));
    op->t_setup[2] = std::chrono::duration<double>(std::chrono::steady_clock::now() - tl0).count();
    op->has_prec = true;
    return LS_OK;
}

// GMRES workspace of an operator with op->nq unknowns and op->prm.max_iter
static ls_status alloc_gmres(ls_op* op, int nsm) {
    const int n = op->nq, maxit = op->prm.max_iter;
    CK(op->Vb.alloc((size_t)(maxit + 1) * n));
    CK(op->Wb.alloc((size_t)maxit * n));
    CK(op->H.alloc((size_t)(maxit + 1) * maxit));
    CK(op->Hraw.alloc((size_t)(maxit + 1) * maxit));
    CK(op->cs.alloc(maxit + 1));
    CK(op->sn.alloc(maxit + 1));
    CK(op->g.alloc(maxit + 2));
    CK(op->hv.alloc(maxit + 1));
    CK(op->yv.alloc(maxit + 1));
    CK(op->tmp.alloc(n));
    CK(op->tmp2.alloc(n));
    CK(op->scal.alloc(4));
    CK(op->hist.alloc(maxit + 2));
    op->dblk = std::max(1, std::min(nsm * 2, (n + RED_TPB - 1) / RED_TPB));
    CK(op->dpart.alloc((size_t)op->dblk * (maxit + 1)));
    return LS_OK;
}

ls_status ls_operator_create(const ls_mesh* mesh, double k, const double* m, const double* m_grid,
                             const ls_params* params, void* stream, ls_op** out) {
    if (!out) return fail(LS_EINVAL, "out is null");
    *out = nullptr;
    if (!mesh || !m) return fail(LS_EINVAL, "null mesh or contrast");
    if (!(k > 0) || !std::isfinite(k)) return fail(LS_EINVAL, "k must be positive");
    ls_params prm;
    ls_params_default(&prm);
    if (params) prm = *params;
    if (prm.max_iter < 1 || !(prm.tol > 0) || !(prm.kappa > 0)) return fail(LS_EINVAL, "bad tol / max_iter / kappa");
    if (prm.prec < 0 || prm.prec > 4)
        return fail(LS_EINVAL, "prec must be 0 (FP64 table), 1 (FP64 direct), 2 (FP32), 3 (double-float) or 4 (mixed)");
    if (prm.approach != 1 && prm.approach != 2) return fail(LS_EINVAL, "approach must be 1 or 2");
    if (prm.use_precond && !m_grid) return fail(LS_EINVAL, "m_grid is required with use_precond");
    const HostMesh& M = mesh->h;
    for (int q = 0; q < M.nq; ++q)
        if (!std::isfinite(m[2 * q]) || !std::isfinite(m[2 * q + 1])) return fail(LS_EINVAL, "non-finite contrast");
    ls_op* op = new (std::nothrow) ls_op;
    if (!op) return fail(LS_ENOMEM, "host allocation");
    struct Guard { ls_op*& p; bool keep = false; ~Guard() { if (!keep) delete p; } } guard{op};
    op->nq = M.nq;
    op->k = k;
    op->prm = prm;
    op->stream = (cudaStream_t)stream;
    const int n = M.nq;
    // correction (host, extended precision)
    auto tc0 = std::chrono::steady_clock::now();
    std::string err = prm.setup_on_device
                          ? lsgpu::build_correction_device(M, k, prm.kappa, stream, op->host_csr, &op->corr_host_blocks)
                          : lsgpu::build_correction(M, k, prm.kappa, op->host_csr);
    op->t_setup[0] = std::chrono::duration<double>(std::chrono::steady_clock::now() - tc0).count();
    if (!err.empty()) return fail(err.find("singular") != std::string::npos ? LS_ESINGULAR : LS_ECUDA, err);
    op->host_nodes = M.nodes;
    op->host_w = M.w;
    CK(op->xy.alloc(n));
    CK(op->w.alloc(n));
    CK(op->m.alloc(n));
    CK(op->rowptr.alloc(n + 1));
    CK(op->cols.alloc(op->host_csr.cols.size()));
    CK(op->vals.alloc(op->host_csr.vals.size()));
    CK(cudaMemcpy(op->xy.p, M.nodes.data(), sizeof(double2) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->w.p, M.w.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->m.p, m, sizeof(double2) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->rowptr.p, op->host_csr.rowptr.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->cols.p, op->host_csr.cols.data(), sizeof(int) * op->host_csr.cols.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(op->vals.p, op->host_csr.vals.data(), sizeof(double2) * op->host_csr.vals.size(), cudaMemcpyHostToDevice));
    {   // dV^T as CSR (rows = source nodes)
        const CsrC& A = op->host_csr;
        const size_t nnz = A.cols.size();
        std::vector<int64_t> rp(n + 1, 0);
        for (size_t e = 0; e < nnz; ++e) rp[A.cols[e] + 1]++;
        for (int i = 0; i < n; ++i) rp[i + 1] += rp[i];
        std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
        std::vector<int> ci(nnz);
        std::vector<std::complex<double>> cv(nnz);
        for (int r = 0; r < n; ++r)
            for (int64_t e = A.rowptr[r]; e < A.rowptr[r + 1]; ++e) {
                int64_t pos = fill[A.cols[e]]++;
                ci[pos] = r;
                cv[pos] = A.vals[e];
            }
        CK(op->rowptrT.alloc(n + 1));
        CK(op->colsT.alloc(nnz));
        CK(op->valsT.alloc(nnz));
        CK(cudaMemcpy(op->rowptrT.p, rp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(op->colsT.p, ci.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(op->valsT.p, cv.data(), sizeof(double2) * nnz, cudaMemcpyHostToDevice));
    }
    // pair-sum decomposition: about 8 resident blocks per SM on 148 SMs
    int dev = 0, nsm = 148;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int tblocks = (n + PS_TPB - 1) / PS_TPB;
    int nchunk = std::max(1, std::min(64, (nsm * 8 + tblocks - 1) / tblocks));
    int spc = (n + nchunk - 1) / nchunk;
    spc = ((spc + PS_TILE - 1) / PS_TILE) * PS_TILE;
    nchunk = (n + spc - 1) / spc;
    op->nchunk = nchunk;
    op->src_per_chunk = spc;
    {   // symmetric decomposition: about 12 CTAs per SM over (strip, distance chunk)
        const int nb = tblocks, D = nb / 2;
        int C = 1, dper = 1;
        if (D > 0) {
            C = std::max(1, std::min(D, (12 * nsm + nb - 1) / nb));
            dper = (D + C - 1) / C;
            C = (D + dper - 1) / dper;
        }
        op->dfs_nb = nb;
        op->dfs_nchunk = C;
        op->dfs_dper = dper;
    }
    CK(op->partial.alloc((size_t)std::max(nchunk, op->dfs_nchunk + op->dfs_nb / 2) * n));
    op->mode = prm.prec;
    op->refine_single = prm.prec == 3 || prm.prec == 4;   // the double-float batched residual is available
    table_range(op, M);
    auto tt0 = std::chrono::steady_clock::now();
    if (prm.prec != 1) TRY(build_table_range(op, op->tab_tlo, op->tab_thi, prm.prec == 4 ? 3 : prm.prec));
    if (prm.prec == 4) TRY(ensure_table32_single(op));
    op->t_setup[3] = std::chrono::duration<double>(std::chrono::steady_clock::now() - tt0).count();
    TRY(alloc_gmres(op, nsm));
    if (prm.use_precond) TRY(build_preconditioner(op, M, m_grid));
    guard.keep = true;
    *out = op;
    return LS_OK;
}

ls_status ls_cartesian_create(double k, const double* m_grid, const ls_params* params, void* stream, ls_op** out) {
    if (!out) return fail(LS_EINVAL, "out is null");
    *out = nullptr;
    if (!m_grid) return fail(LS_EINVAL, "null contrast");
    if (!(k > 0) || !std::isfinite(k)) return fail(LS_EINVAL, "k must be positive");
    ls_params prm;
    ls_params_default(&prm);
    if (params) prm = *params;
    if (prm.max_iter < 1 || !(prm.tol > 0)) return fail(LS_EINVAL, "bad tol / max_iter");
    const int nx = prm.nx, ny = prm.ny;
    if (nx < 4 || ny < 4) return fail(LS_EINVAL, "grid needs at least 4 x 4 nodes");
    const double h = (prm.box[1] - prm.box[0]) / (nx - 1);
    if (!(h > 0) || std::fabs((prm.box[3] - prm.box[2]) / (ny - 1) - h) > 1e-12 * h)
        return fail(LS_EINVAL, "grid step must be equal in x and y");
    const int n = nx * ny;
    for (int q = 0; q < n; ++q)
        if (!std::isfinite(m_grid[2 * q]) || !std::isfinite(m_grid[2 * q + 1])) return fail(LS_EINVAL, "non-finite contrast");
    ls_op* op = new (std::nothrow) ls_op;
    if (!op) return fail(LS_ENOMEM, "host allocation");
    struct Guard { ls_op*& p; bool keep = false; ~Guard() { if (!keep) delete p; } } guard{op};
    op->cartesian = true;
    op->nq = n;
    op->k = k;
    op->prm = prm;
    op->stream = (cudaStream_t)stream;
    op->nx = nx;
    op->ny = ny;
    int dev = 0, nsm = 148;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    {   // unknowns at the grid nodes (x fastest), weights h^2 for the far field
        std::vector<double2> xy(n);
        std::vector<double> w(n, h * h);
        for (int b = 0; b < ny; ++b)
            for (int a = 0; a < nx; ++a) xy[a + (size_t)nx * b] = make_double2(prm.box[0] + a * h, prm.box[2] + b * h);
        CK(op->xy.alloc(n));
        CK(op->w.alloc(n));
        CK(op->m.alloc(n));
        CK(cudaMemcpy(op->xy.p, xy.data(), sizeof(double2) * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(op->w.p, w.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(op->m.p, m_grid, sizeof(double2) * n, cudaMemcpyHostToDevice));
    }
    auto tt0 = std::chrono::steady_clock::now();
    {   // spectrum of the zero-padded kernel, scaled by 1 / (NX NY) for the inverse transform
        op->cNX = 2 * nx;
        op->cNY = 2 * ny;
        const int NX = op->cNX, NY = op->cNY;
        std::vector<std::complex<double>> tab;
        lsgpu::cartesian_kernel_table(k, h, nx, ny, tab);
        const double sc = 1.0 / ((double)NX * NY);
        for (auto& v : tab) v *= sc;
        DevBuf<double2> dtab;
        CK(dtab.alloc(tab.size()));
        CK(cudaMemcpy(dtab.p, tab.data(), sizeof(double2) * tab.size(), cudaMemcpyHostToDevice));
        CK(op->khat.alloc((size_t)NX * NY));
        CK(op->fpad.alloc((size_t)NX * NY));
        CK(op->czero.alloc(n));
        CK(cudaMemsetAsync(op->czero.p, 0, sizeof(double2) * n, op->stream));
        k_cart_kernel<<<dim3((NX + 127) / 128, NY), 128, 0, op->stream>>>(nx, ny, NX, NY, dtab.p, op->khat.p);
        CK(cudaGetLastError());
        if (cufftPlan2d(&op->fft, NY, NX, CUFFT_Z2Z) != CUFFT_SUCCESS) return fail(LS_ECUDA, "cufftPlan2d failed");
        if (cufftSetStream(op->fft, op->stream) != CUFFT_SUCCESS) return fail(LS_ECUDA, "cufftSetStream failed");
        if (cufftExecZ2Z(op->fft, (cufftDoubleComplex*)op->khat.p, (cufftDoubleComplex*)op->khat.p, CUFFT_FORWARD) !=
            CUFFT_SUCCESS)
            return fail(LS_ECUDA, "cufftExecZ2Z failed");
        CK(cudaStreamSynchronize(op->stream));
    }
    op->t_setup[3] = std::chrono::duration<double>(std::chrono::steady_clock::now() - tt0).count();
    TRY(alloc_gmres(op, nsm));
    if (prm.use_precond) {
        auto tg0 = std::chrono::steady_clock::now();
        GridSetup G;
        std::vector<std::complex<double>> mg(n);
        for (int i = 0; i < n; ++i) mg[i] = std::complex<double>(m_grid[2 * i], m_grid[2 * i + 1]);
        std::string err = lsgpu::build_stencil_C(k, prm.box, nx, ny, mg.data(), G);
        if (!err.empty()) return fail(LS_EINVAL, err);
        op->t_setup[1] = std::chrono::duration<double>(std::chrono::steady_clock::now() - tg0).count();
        auto tl0 = std::chrono::steady_clock::now();
        std::vector<double2> hs(81);
        for (int c = 0; c < 9; ++c)
            for (int t = 0; t < 9; ++t) hs[9 * c + t] = make_double2(G.v[c][t].real(), G.v[c][t].imag());
        CK(op->st.alloc(81));
        CK(cudaMemcpy(op->st.p, hs.data(), sizeof(double2) * 81, cudaMemcpyHostToDevice));
        CK(op->cband.alloc(G.cband.size()));
        CK(cudaMemcpy(op->cband.p, G.cband.data(), sizeof(double2) * G.cband.size(), cudaMemcpyHostToDevice));
        CK(op->ptp.alloc(n));
        TRY(build_cr(op));
        op->t_setup[2] = std::chrono::duration<double>(std::chrono::steady_clock::now() - tl0).count();
        op->has_prec = true;
    }
    guard.keep = true;
    *out = op;
    return LS_OK;
}

void ls_op_destroy(ls_op* op) { delete op; }

ls_status ls_apply_dev(ls_op* op, const void* x_dev, void* y_dev) {
    if (!op || !x_dev || !y_dev) return fail(LS_EINVAL, "null argument");
    if (x_dev == y_dev) return fail(LS_EINVAL, "x and y may not alias");
    TRY(apply_L(op, (const double2*)x_dev, (double2*)y_dev));
    return check_stream_sync(op);
}

ls_status ls_apply(ls_op* op, const double* x, double* y) {
    if (!op || !x || !y) return fail(LS_EINVAL, "null argument");
    CK(cudaMemcpyAsync(op->tmp.p, x, sizeof(double2) * op->nq, cudaMemcpyHostToDevice, op->stream));
    TRY(apply_L(op, op->tmp.p, op->tmp2.p));
    CK(cudaMemcpyAsync(y, op->tmp2.p, sizeof(double2) * op->nq, cudaMemcpyDeviceToHost, op->stream));
    return check_stream_sync(op);
}

ls_status ls_apply_precond_dev(ls_op* op, const void* x_dev, void* y_dev) {
    if (!op || !x_dev || !y_dev) return fail(LS_EINVAL, "null argument");
    if (!op->has_prec) return fail(LS_EINVAL, "operator was built without a preconditioner");
    if (x_dev == y_dev) return fail(LS_EINVAL, "x and y may not alias");
    TRY(apply_P(op, (const double2*)x_dev, (double2*)y_dev));
    return check_stream_sync(op);
}

ls_status ls_pairsum_dev(ls_op* op, const void* f_dev, void* y_dev) {
    if (!op || !f_dev || !y_dev) return fail(LS_EINVAL, "null argument");
    TRY(launch_pairsum(op, (const double2*)f_dev, nullptr));
    TRY(collapse_slots(op));
    int threads = 256;
    int blocks = (int)(((int64_t)op->nq * 32 + threads - 1) / threads);
    k_apply_epi<<<blocks, threads, 0, op->stream>>>(op->nq, op->ps_slots, op->partial.p, op->rowptr.p, op->cols.p,
                                                    op->vals.p, op->m.p, (const double2*)f_dev, 0.0, (double2*)y_dev, 1);
    CK(cudaGetLastError());
    return check_stream_sync(op);
}

static ls_status farfield(ls_op* op, const double2* u, int n_ff, const double* ang_dev, double2* out_dev) {
    k_farfield<<<n_ff, RED_TPB, 0, op->stream>>>(op->nq, op->xy.p, op->w.p, op->m.p, u, op->k, ang_dev, out_dev);
    CK(cudaGetLastError());
    op->launches++;
    return LS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batched form (host side)
static ls_status ensure_batch(ls_op* op, int R) {
    if (op->cartesian) return fail(LS_EINVAL, "the batched forms need a quadrature-node operator");
    if (op->bR >= R) return LS_OK;
    const int n = op->nq, maxit = op->prm.max_iter, ldh = maxit + 1;
    int dev = 0, nsm = 148;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int tblocks = (n + PS_TPB - 1) / PS_TPB, rblocks = (R + MRB - 1) / MRB;
    int nchunk = std::max(1, std::min(16, (nsm * 4 + tblocks * rblocks - 1) / (tblocks * rblocks)));
    int spc = (n + nchunk - 1) / nchunk;
    spc = ((spc + PS_TILE - 1) / PS_TILE) * PS_TILE;
    op->b_nchunk = (n + spc - 1) / spc;
    op->b_spc = spc;
    {
        // tensor-core form: units (128-target tile, source chunk) taken round-robin by one
        // resident CTA per SM; about 8 units per SM, chunks a multiple of 16 sources
        const int tb = (n + TC_M - 1) / TC_M;
        int nc = std::max(1, std::min(32, (8 * nsm + tb - 1) / tb));
        int tspc = (n + nc - 1) / nc;
        tspc = ((tspc + TC_SRC - 1) / TC_SRC) * TC_SRC;
        op->tc_spc = tspc;
        op->tc_nchunk = (n + tspc - 1) / tspc;
    }
    CK(op->bV.alloc((size_t)R * (maxit + 1) * n));
    CK(op->bH.alloc((size_t)R * ldh * maxit));
    CK(op->bcs.alloc((size_t)R * (maxit + 2)));
    CK(op->bsn.alloc((size_t)R * (maxit + 2)));
    CK(op->bg.alloc((size_t)R * (maxit + 2)));
    CK(op->bhv.alloc((size_t)R * (maxit + 1)));
    CK(op->byv.alloc((size_t)R * (maxit + 1)));
    CK(op->btmp.alloc((size_t)R * n));
    CK(op->bdpart.alloc((size_t)R * (maxit + 1) * op->dblk));
    CK(op->bscal.alloc((size_t)2 * R));
    CK(op->bpartial.alloc((size_t)R * std::max(op->b_nchunk, op->tc_nchunk) * n));
    CK(op->bhist.alloc((size_t)R * (maxit + 2)));
    CK(op->bactive.alloc(R));
    CK(op->bits.alloc(R));
    if (op->has_prec) {
        const size_t nc = (size_t)op->nx * op->ny;
        CK(op->bpg.alloc(R * nc));
        CK(op->bpt.alloc(R * nc));
        CK(op->bptp.alloc(R * nc));
    }
    op->bR = R;
    return LS_OK;
}

static MultiArgs multi_args(ls_op* op, int R, const double2* f, size_t sf, const double2* m) {
    MultiArgs A;
    A.xy = op->xy.p; A.w = op->w.p; A.m = m; A.f = f; A.sf = sf;
    A.n = op->nq; A.R = R; A.spc = op->b_spc; A.nchunk = op->b_nchunk;
    A.k = op->k; A.inv_k = 1.0 / op->k;
    A.ncell = op->t32_ncell; A.noct = op->t32_noct; A.b_lo = op->t32_blo;
    A.partial = op->bpartial.p;
    return A;
}

// partial[r][c][j] for R densities f (stride sf); w = nullptr takes unit weights
static ls_status pairsum_batch(ls_op* op, int R, const double2* f, size_t sf, const double2* m, const double* w);
static ls_status pairsum_batch(ls_op* op, int R, const double2* f, size_t sf, const double2* m) {
    return pairsum_batch(op, R, f, sf, m, op->w.p);
}
static ls_status ensure_tc(ls_op* op) {
    if (op->tc_herr) return LS_OK;
    const int n = op->nq;
    op->tc_npad = ((n + TC_SRC - 1) / TC_SRC) * TC_SRC;
    CK(op->tc_xy32.alloc(op->tc_npad));
    CK(op->tc_Sc.alloc((size_t)op->tc_npad * 64));
    CK(op->tc_err.alloc(1));
    CK(cudaMemsetAsync(op->tc_err.p, 0, sizeof(int), op->stream));
    k_tc_xy32<<<(op->tc_npad + 255) / 256, 256, 0, op->stream>>>(n, op->tc_npad, op->xy.p, op->tc_xy32.p);
    CK(cudaGetLastError());
    CK(op->tc_desc.alloc(TC_MAX_OPS));
    CK(cudaMallocHost(&op->tc_herr, sizeof(int)));
    *op->tc_herr = 0;
    return LS_OK;
}

static size_t tc_smem_bytes(int N, size_t tab_bytes, int nstg) {
    const size_t stage = 2 * (size_t)TC_M * 2 * TC_SRC * 4 + 2 * (size_t)N * 2 * TC_SRC * 4;
    const size_t stg = (size_t)TC_SRC * (N / 2) * 16 + TC_SRC * 16;
    return 1024 + TC_NS * stage + (size_t)nstg * stg + tab_bytes;
}

static TCOp tc_desc_of(ls_op* op, int unit_begin) {
    TCOp o;
    o.xy32 = op->tc_xy32.p;
    o.Sc = op->tc_Sc.p;
    o.tab = (const float4*)op->tab32.p;
    o.partial = op->bpartial.p;
    o.k = op->k;
    o.inv_k = 1.0 / op->k;
    o.n = op->nq;
    o.tblocks = (op->nq + TC_M - 1) / TC_M;
    o.spc = op->tc_spc;
    o.nchunk = op->tc_nchunk;
    o.part_nchunk = op->tc_nchunk;
    o.unit_begin = unit_begin;
    o.units = o.tblocks * o.nchunk;
    o.ncell = op->t32_ncell;
    o.noct = op->t32_noct;
    o.b_lo = op->t32_blo;
    o.tab_words = (int)(op->t32_bytes / sizeof(float4));
    return o;
}

// One tensor-core pair sum over S operators (each with R right-hand sides f_s, stride
// sf_s), groups of up to 64 right-hand sides per launch; partials [R][tc_nchunk][n] per
// operator.  desc: device array of S descriptors (rewritten here).
static ls_status pairsum_tc_launch(int S, ls_op* const* ops, int R, const double2* const* f, const size_t* sf,
                                   const double2* const* m, const double* const* w, TCOp* desc,
                                   std::vector<TCOp>& host_desc, cudaStream_t st) {
    int dev = 0, nsm = 148;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (S > TC_MAX_OPS) return fail(LS_EINVAL, "too many operators for one tensor-core launch");
    std::vector<TCOp> d(S);
    int total = 0;
    size_t max_tab = 0;
    for (int s = 0; s < S; ++s) {
        d[s] = tc_desc_of(ops[s], total);
        total += d[s].units;
        max_tab = std::max(max_tab, ops[s]->t32_bytes);
    }
    // upload only when the descriptors changed (a pageable copy may synchronise the stream)
    if (host_desc.size() != d.size() || std::memcmp(host_desc.data(), d.data(), sizeof(TCOp) * S) != 0) {
        CK(cudaMemcpy(desc, d.data(), sizeof(TCOp) * S, cudaMemcpyHostToDevice));
        host_desc = d;
    }
    for (int r0 = 0; r0 < R; r0 += 64) {
        const int Rg = std::min(64, R - r0);
        int Rp = 8;
        while (Rp < Rg) Rp *= 2;
        const int N = 2 * Rp;
        for (int s = 0; s < S; ++s) {
            ls_op* op = ops[s];
            const int64_t tot = (int64_t)op->tc_npad * Rp;
            k_tc_prep_S<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(op->nq, op->tc_npad, Rg, Rp, f[s] + (size_t)r0 * sf[s],
                                                                     sf[s], w[s], m[s], op->tc_Sc.p);
            op->launches++;
        }
        CK(cudaGetLastError());
        TCArgs A;
        A.ops = desc;
        A.S = S;
        A.total_units = total;
        A.R = Rg; A.Rp = Rp; A.N = N;
        A.F = std::max(1, ops[0]->tc_fold);
        A.r_offset = r0;
        A.idesc = tc::idesc_tf32(TC_M, N);
        A.err = ops[0]->tc_err.p;
        A.stall_ns = ops[0]->tc_stall_ns;
        // three staging slots when they fit beside the table, else two
        A.nstg = tc_smem_bytes(N, max_tab, 3) <= 227 * 1024 ? 3 : 2;
        const size_t smem = tc_smem_bytes(N, max_tab, A.nstg);
        if (smem > 227 * 1024) return fail(LS_EINVAL, "H0 table too large for the tensor-core pair sum");
        CK(raise_smem_limit(k_pairsum_tc, smem));
        k_pairsum_tc<<<std::min(total, nsm), TC_THREADS, smem, st>>>(A);
        CK(cudaGetLastError());
        ops[0]->launches++;
    }
    CK(cudaMemcpyAsync(ops[0]->tc_herr, ops[0]->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    for (int s = 0; s < S; ++s) ops[s]->b_nchunk_cur = ops[s]->tc_nchunk;
    return LS_OK;
}

// Tensor-core form of pairsum_batch for one operator.
static ls_status pairsum_batch_tc(ls_op* op, int R, const double2* f, size_t sf, const double2* m, const double* w) {
    TRY(ensure_tc(op));
    ls_op* ops[1] = {op};
    const double2* fs[1] = {f};
    const size_t sfs[1] = {sf};
    const double2* ms[1] = {m};
    const double* ws[1] = {w};
    return pairsum_tc_launch(1, ops, R, fs, sfs, ms, ws, op->tc_desc.p, op->tc_hdesc, op->stream);
}

// error word of the tensor-core pair sum, read after a stream synchronisation
// (the word is cleared on report, so the operator stays usable for the next call)
static ls_status tc_status(ls_op* op) {
    if (op->tc_herr && *op->tc_herr) {
        const int code = *op->tc_herr;
        *op->tc_herr = 0;
        CK(cudaMemsetAsync(op->tc_err.p, 0, sizeof(int), op->stream));
        CK(cudaStreamSynchronize(op->stream));
        return fail(LS_ETIMEOUT, "tensor-core pair sum: a pipeline wait ran out (code " + std::to_string(code) + ")");
    }
    return LS_OK;
}

static ls_status pairsum_batch_df(ls_op* op, int R, const double2* f, size_t sf, const double2* m, const double* w);

static ls_status pairsum_batch(ls_op* op, int R, const double2* f, size_t sf, const double2* m, const double* w) {
    if (op->batch_kernel == 2) return pairsum_batch_df(op, R, f, sf, m, w);
    TRY(ensure_table32(op));
    if (op->batch_kernel == 1) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (op->timing && op->ev.size() < 65536) {
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            op->ev.emplace_back(e0, e1);
            op->ev_kind.push_back(11);
            CK(cudaEventRecord(e0, op->stream));
        }
        TRY(pairsum_batch_tc(op, R, f, sf, m, w));
        if (e1) CK(cudaEventRecord(e1, op->stream));
        op->pairsum_launches++;
        return LS_OK;
    }
    op->b_nchunk_cur = op->b_nchunk;
    dim3 grid((op->nq + PS_TPB - 1) / PS_TPB, op->b_nchunk, (R + MRB - 1) / MRB);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (op->timing && op->ev.size() < 65536) {
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        op->ev.emplace_back(e0, e1);
        op->ev_kind.push_back(10);
        CK(cudaEventRecord(e0, op->stream));
    }
    MultiArgs A = multi_args(op, R, f, sf, m);
    A.w = w;
    k_pairsum_multi_f32<<<grid, PS_TPB, op->t32_bytes, op->stream>>>(A, (const float4*)op->tab32.p);
    CK(cudaGetLastError());
    if (e1) CK(cudaEventRecord(e1, op->stream));
    op->launches++;
    op->pairsum_launches++;
    return LS_OK;
}

// FP32 copies of the block-LU factors and of the band of C, and the FP32 sweep vectors.
static ls_status ensure_sweeps32(ls_op* op, int R) {
    const size_t nx = op->nx, ny = op->ny, nc = nx * ny;
    if (!op->Wf32.p) {
        const int64_t nf = (int64_t)(ny * nx * nx), nb = (int64_t)(ny * 9 * nx);
        CK(op->Wf32.alloc(nf));
        CK(op->Gf32.alloc(nf));
        CK(op->cband32.alloc(nb));
        k_to_f32<<<(unsigned)((nf + 255) / 256), 256, 0, op->stream>>>(nf, op->Wf.p, op->Wf32.p);
        k_to_f32<<<(unsigned)((nf + 255) / 256), 256, 0, op->stream>>>(nf, op->Gf.p, op->Gf32.p);
        k_to_f32<<<(unsigned)((nb + 255) / 256), 256, 0, op->stream>>>(nb, op->cband.p, op->cband32.p);
        CK(cudaGetLastError());
        op->launches += 3;
    }
    if (op->by32.n < (size_t)R * nc) CK(op->by32.alloc((size_t)R * nc));
    return LS_OK;
}

static ls_status apply_P_batch(ls_op* op, int R, const double2* x, size_t sx, double2* z, size_t sz) {
    const int nx = op->nx, ny = op->ny, nc = nx * ny;
    dim3 gc((nc + 255) / 256, R);
    k_tqc_multi<<<gc, 256, 0, op->stream>>>(nc, op->tqc_rp.p, op->tqc_ci.p, op->tqc_cv.p, x, sx, op->bpg.p);
    k_stencil_multi<<<gc, 256, 0, op->stream>>>(nx, ny, op->st.p, op->bpg.p, op->bpt.p);
    if (op->batch_kernel == 1) {
        // tensor-core form: FP32 sweeps (the solve is refined against the accurate operator)
        TRY(ensure_sweeps32(op, R));
        dim3 gs((nx + BT_ROWS - 1) / BT_ROWS, (R + BT_RHS - 1) / BT_RHS);
        for (int b = 0; b < ny; ++b)
            k_bt_sweep32<<<gs, 256, 0, op->stream>>>(nx, ny, b, R, 0, op->Wf32.p, op->cband32.p, op->bpt.p,
                                                     op->by32.p);
        for (int b = ny - 2; b >= 0; --b)
            k_bt_sweep32<<<gs, 256, 0, op->stream>>>(nx, ny, b, R, 1, op->Gf32.p, nullptr, nullptr, op->by32.p);
        const int64_t tot = (int64_t)R * nc;
        k_to_f64<<<(unsigned)((tot + 255) / 256), 256, 0, op->stream>>>(tot, op->by32.p, op->bptp.p);
        op->launches += 1;
    } else {
        const int wpb = 8;
        dim3 gb((nx + wpb - 1) / wpb, R);
        const size_t shm = sizeof(double2) * nx;
        for (int b = 0; b < ny; ++b)
            k_bt_fwd_multi<<<gb, 32 * wpb, shm, op->stream>>>(nx, ny, b, op->Wf.p, op->cband.p, op->bpt.p, op->bptp.p);
        for (int b = ny - 2; b >= 0; --b)
            k_bt_bwd_multi<<<gb, 32 * wpb, shm, op->stream>>>(nx, ny, b, op->Gf.p, op->bptp.p);
    }
    dim3 gq((op->nq + 255) / 256, R);
    k_tcq_multi<<<gq, 256, 0, op->stream>>>(op->nq, nc, op->tcq_idx.p, op->tcq_w.p, op->bptp.p, op->bpg.p, x, sx, z, sz);
    CK(cudaGetLastError());
    op->launches += 3 + ny + (ny - 1);
    return LS_OK;
}

static ls_status apply_PT_batch(ls_op* op, int R, const double2* x, size_t sx, double2* z, size_t sz) {
    const int nx = op->nx, ny = op->ny, nc = nx * ny;
    dim3 gc((nc + 255) / 256, R);
    k_tqc_multi<<<gc, 256, 0, op->stream>>>(nc, op->tcqT_rp.p, op->tcqT_ci.p, op->tcqT_cv.p, x, sx, op->bpg.p);
    CK(cudaMemcpyAsync(op->bptp.p, op->bpg.p, sizeof(double2) * R * nc, cudaMemcpyDeviceToDevice, op->stream));
    const int wpb = 8;
    dim3 gb((nx + wpb - 1) / wpb, R);
    const size_t shm = sizeof(double2) * nx;
    for (int b = 1; b < ny; ++b)
        k_btT_fwd_multi<<<gb, 32 * wpb, shm, op->stream>>>(nx, ny, b, op->GT.p, op->bptp.p);
    for (int b = ny - 1; b >= 0; --b)
        k_btT_bwd_multi<<<gb, 32 * wpb, shm, op->stream>>>(nx, ny, b, op->WT.p, op->cband.p, op->bptp.p, op->bpt.p);
    k_stencilT_multi<<<gc, 256, 0, op->stream>>>(nx, ny, op->st.p, op->bpt.p, op->bpg.p, op->bptp.p);
    dim3 gq((op->nq + 255) / 256, R);
    k_tqcT<<<gq, 256, 0, op->stream>>>(op->nq, op->tqcT_rp.p, op->tqcT_ci.p, op->tqcT_cv.p, op->bptp.p, nc, x, sx, z, sz);
    CK(cudaGetLastError());
    op->launches += 3 + (ny - 1) + ny;
    return LS_OK;
}

// R lock-step GMRES solves (each system its own Krylov space, Hessenberg and stop),
// split in stages so that several operators can share one pair-sum launch.
static ls_status gb_begin(ls_op* op, int R, const double2* b, bool transpose = false) {
    TRY(ensure_batch(op, R));
    const int n = op->nq, maxit = op->prm.max_iter, ldh = maxit + 1;
    const size_t ldv = (size_t)n, svr = (size_t)(maxit + 1) * n, sH = (size_t)ldh * maxit, sg = maxit + 2;
    const bool prec = op->has_prec && op->prm.use_precond;
    const int tpb = 256, nb = (n + tpb - 1) / tpb;
    CK(cudaMemsetAsync(op->bH.p, 0, sizeof(double2) * R * sH, op->stream));
    if (prec && transpose) TRY(apply_PT_batch(op, R, b, n, op->btmp.p, n));
    else if (prec) TRY(apply_P_batch(op, R, b, n, op->btmp.p, n));
    else CK(cudaMemcpyAsync(op->btmp.p, b, sizeof(double2) * R * n, cudaMemcpyDeviceToDevice, op->stream));
    dim3 gd(op->dblk, R), gn(nb, R);
    k_dots_multi<<<gd, RED_TPB, 0, op->stream>>>(n, 1, op->btmp.p, n, ldv, op->btmp.p, n, op->bdpart.p, nullptr);
    k_sumrows_multi<<<dim3(1, R), 128, 0, op->stream>>>(1, op->dblk, op->bdpart.p, op->bscal.p, 1, 0, nullptr);
    k_scale_multi<<<gn, tpb, 0, op->stream>>>(n, op->btmp.p, n, op->bscal.p, op->bV.p, svr, nullptr, 0, nullptr);
    k_gmres_init_multi<<<(R + 127) / 128, 128, 0, op->stream>>>(R, op->bg.p, sg, op->bscal.p, op->bhist.p, sg,
                                                                op->bactive.p, op->bits.p);
    CK(cudaGetLastError());
    op->launches += 4;
    return LS_OK;
}

// Everything of iteration j after the pair sum (partials in op->bpartial).
static ls_status gb_after_pairsum(ls_op* op, int R, int j, bool transpose = false) {
    const int n = op->nq, maxit = op->prm.max_iter, ldh = maxit + 1;
    const size_t ldv = (size_t)n, svr = (size_t)(maxit + 1) * n, sH = (size_t)ldh * maxit, sg = maxit + 2;
    const bool prec = op->has_prec && op->prm.use_precond;
    const int tpb = 256, nb = (n + tpb - 1) / tpb;
    double2* V = op->bV.p;
    double2* vj = V + (size_t)j * ldv;
    double2* vn = V + (size_t)(j + 1) * ldv;
    double2* hcol = op->bH.p + (size_t)j * ldh;
    dim3 ge((unsigned)(((int64_t)n * 32 + 255) / 256), R);
    if (transpose)
        k_applyT_epi_multi<<<ge, 256, 0, op->stream>>>(n, op->b_nchunk_cur, op->bpartial.p, op->rowptrT.p, op->colsT.p,
                                                       op->valsT.p, op->m.p, op->w.p, vj, svr, op->k * op->k,
                                                       prec ? op->btmp.p : vn, prec ? (size_t)n : svr);
    else
        k_apply_epi_multi<<<ge, 256, 0, op->stream>>>(n, op->b_nchunk_cur, op->bpartial.p, op->rowptr.p, op->cols.p, op->vals.p,
                                                      op->m.p, vj, svr, op->k * op->k, prec ? op->btmp.p : vn,
                                                      prec ? (size_t)n : svr);
    op->launches++;
    if (prec && transpose) TRY(apply_PT_batch(op, R, op->btmp.p, n, vn, svr));
    else if (prec) TRY(apply_P_batch(op, R, op->btmp.p, n, vn, svr));
    const int J = j + 1;
    dim3 gd(op->dblk, R), gn(nb, R), gs((J + 127) / 128, R);
    k_dots_multi<<<gd, RED_TPB, 0, op->stream>>>(n, J, V, svr, ldv, vn, svr, op->bdpart.p, op->bactive.p);
    k_sumrows_multi<<<gs, 128, 0, op->stream>>>(J, op->dblk, op->bdpart.p, hcol, sH, 0, op->bactive.p);
    k_update_multi<<<gn, tpb, sizeof(double2) * J, op->stream>>>(n, J, V, svr, ldv, hcol, sH, vn, svr, op->bactive.p);
    k_dots_multi<<<gd, RED_TPB, 0, op->stream>>>(n, J, V, svr, ldv, vn, svr, op->bdpart.p, op->bactive.p);
    k_sumrows_multi<<<gs, 128, 0, op->stream>>>(J, op->dblk, op->bdpart.p, op->bhv.p, J, 0, op->bactive.p);
    k_update_multi<<<gn, tpb, sizeof(double2) * J, op->stream>>>(n, J, V, svr, ldv, op->bhv.p, J, vn, svr, op->bactive.p);
    k_sumrows_multi<<<gs, 128, 0, op->stream>>>(J, 1, op->bhv.p, hcol, sH, 1, op->bactive.p);
    k_dots_multi<<<gd, RED_TPB, 0, op->stream>>>(n, 1, vn, svr, ldv, vn, svr, op->bdpart.p, op->bactive.p);
    k_sumrows_multi<<<dim3(1, R), 128, 0, op->stream>>>(1, op->dblk, op->bdpart.p, op->bscal.p + R, 1, 0, op->bactive.p);
    k_scale_multi<<<gn, tpb, 0, op->stream>>>(n, vn, svr, op->bscal.p + R, vn, svr, hcol + j + 1, sH, op->bactive.p);
    k_givens_multi<<<(R + 127) / 128, 128, 0, op->stream>>>(R, j, op->bH.p, sH, ldh, op->bcs.p, op->bsn.p, op->bg.p, sg,
                                                            op->bhist.p, sg, op->bscal.p, op->prm.tol, op->bactive.p,
                                                            op->bits.p);
    CK(cudaGetLastError());
    op->launches += 11;
    return LS_OK;
}

static ls_status gb_active(ls_op* op, int R, std::vector<int>& act, bool& any) {
    act.resize(R);
    CK(cudaMemcpyAsync(act.data(), op->bactive.p, sizeof(int) * R, cudaMemcpyDeviceToHost, op->stream));
    CK(cudaStreamSynchronize(op->stream));
    TRY(tc_status(op));
    any = false;
    for (int r = 0; r < R; ++r) any = any || act[r];
    return LS_OK;
}

static ls_status gb_finish(ls_op* op, int R, double2* u, int* iters, bool& all_conv) {
    const int n = op->nq, maxit = op->prm.max_iter, ldh = maxit + 1;
    const size_t ldv = (size_t)n, svr = (size_t)(maxit + 1) * n, sH = (size_t)ldh * maxit, sg = maxit + 2;
    const int tpb = 256, nb = (n + tpb - 1) / tpb;
    k_backsolve_multi<<<(R + 127) / 128, 128, 0, op->stream>>>(R, op->bits.p, op->bH.p, sH, ldh, op->bg.p, sg, op->byv.p,
                                                               maxit + 1);
    k_combine_multi<<<dim3(nb, R), tpb, 0, op->stream>>>(n, op->bits.p, op->bV.p, svr, ldv, op->byv.p, maxit + 1, u, n);
    CK(cudaGetLastError());
    op->launches += 2;
    std::vector<int> its(R), act;
    bool any = false;
    TRY(gb_active(op, R, act, any));
    CK(cudaMemcpyAsync(its.data(), op->bits.p, sizeof(int) * R, cudaMemcpyDeviceToHost, op->stream));
    CK(cudaStreamSynchronize(op->stream));
    for (int r = 0; r < R; ++r)
        if (iters) iters[r] = its[r];
    all_conv = !any;
    return LS_OK;
}

static ls_status gmres_batch_plain(ls_op* op, int R, const double2* b, double2* u, int* iters, bool transpose) {
    TRY(gb_begin(op, R, b, transpose));
    const size_t svr = (size_t)(op->prm.max_iter + 1) * op->nq;
    std::vector<int> act;
    for (int j = 0; j < op->prm.max_iter; ++j) {
        if (transpose) TRY(pairsum_batch(op, R, op->bV.p + (size_t)j * op->nq, svr, nullptr, nullptr));
        else TRY(pairsum_batch(op, R, op->bV.p + (size_t)j * op->nq, svr, op->m.p));
        TRY(gb_after_pairsum(op, R, j, transpose));
        bool any = false;
        TRY(gb_active(op, R, act, any));
        if (!any) break;
    }
    bool all = false;
    TRY(gb_finish(op, R, u, iters, all));
    return all ? LS_OK : LS_ENOCONV;
}

// ||P x_r||^2 for R systems (P^T for the transposed problem) into host nrm2[R]
static ls_status prec_norms(ls_op* op, int R, const double2* x, bool transpose, std::vector<double>& nrm2) {
    const int n = op->nq;
    const bool prec = op->has_prec && op->prm.use_precond;
    const double2* z = x;
    if (prec && transpose) { TRY(apply_PT_batch(op, R, x, n, op->ir_y.p, n)); z = op->ir_y.p; }
    else if (prec) { TRY(apply_P_batch(op, R, x, n, op->ir_y.p, n)); z = op->ir_y.p; }
    dim3 gd(op->dblk, R);
    k_dots_multi<<<gd, RED_TPB, 0, op->stream>>>(n, 1, z, n, n, z, n, op->bdpart.p, nullptr);
    k_sumrows_multi<<<dim3(1, R), 128, 0, op->stream>>>(1, op->dblk, op->bdpart.p, op->bscal.p, 1, 0, nullptr);
    CK(cudaGetLastError());
    op->launches += 2;
    std::vector<double2> h(R);
    CK(cudaMemcpyAsync(h.data(), op->bscal.p, sizeof(double2) * R, cudaMemcpyDeviceToHost, op->stream));
    CK(cudaStreamSynchronize(op->stream));
    nrm2.resize(R);
    for (int r = 0; r < R; ++r) nrm2[r] = h[r].x;
    return LS_OK;
}

// Batched double-float pair sum (k_pairsum_multi_df) on the operator's double-float table.
static ls_status pairsum_batch_df(ls_op* op, int R, const double2* f, size_t sf, const double2* m, const double* w) {
    TRY(ensure_batch(op, R));
    op->b_nchunk_cur = op->b_nchunk;
    dim3 grid((op->nq + PS_TPB - 1) / PS_TPB, op->b_nchunk, (R + MRB - 1) / MRB);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (op->timing && op->ev.size() < 65536) {
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        op->ev.emplace_back(e0, e1);
        op->ev_kind.push_back(12);
        CK(cudaEventRecord(e0, op->stream));
    }
    MultiArgs A;
    A.xy = op->xy.p; A.w = w; A.m = m; A.f = f; A.sf = sf;
    A.n = op->nq; A.R = R; A.spc = op->b_spc; A.nchunk = op->b_nchunk;
    A.k = op->k; A.inv_k = 1.0 / op->k;
    A.ncell = op->tab_ncell; A.noct = op->tab_noct; A.b_lo = op->tab_blo;
    A.partial = op->bpartial.p;
    launch_multi_df(op->tab_nc, op->tab_nf, grid, op->tab_bytes, op->stream, A, (const float4*)op->tab.p);
    CK(cudaGetLastError());
    if (e1) CK(cudaEventRecord(e1, op->stream));
    op->launches++;
    op->pairsum_launches++;
    return LS_OK;
}

// y_r = L x_r (or L^T x_r) with the accurate batched pair sum (CUDA cores, Kahan FP32)
static ls_status apply_L_batch_accurate(ls_op* op, int R, const double2* x, double2* y, bool transpose) {
    const int n = op->nq;
    if (op->refine_single && (op->mode == 3 || op->mode == 4)) {
        // double-float operator: the batched double-float pair sum over all R systems
        TRY(pairsum_batch_df(op, R, x, n, transpose ? nullptr : op->m.p, transpose ? nullptr : op->w.p));
        dim3 ge((unsigned)(((int64_t)n * 32 + 255) / 256), R);
        if (transpose)
            k_applyT_epi_multi<<<ge, 256, 0, op->stream>>>(n, op->b_nchunk_cur, op->bpartial.p, op->rowptrT.p,
                                                           op->colsT.p, op->valsT.p, op->m.p, op->w.p, x, n,
                                                           op->k * op->k, y, n);
        else
            k_apply_epi_multi<<<ge, 256, 0, op->stream>>>(n, op->b_nchunk_cur, op->bpartial.p, op->rowptr.p, op->cols.p,
                                                          op->vals.p, op->m.p, x, n, op->k * op->k, y, n);
        CK(cudaGetLastError());
        op->launches++;
        return LS_OK;
    }
    if (op->refine_single) {
        // the operator's own single-RHS pair sum, one system at a time (FP64-accurate with the
        // FP64 forms)
        for (int r = 0; r < R; ++r) {
            const double2* xr = x + (size_t)r * n;
            double2* yr = y + (size_t)r * n;
            TRY(transpose ? apply_LT(op, xr, yr) : apply_L(op, xr, yr));
        }
        return LS_OK;
    }
    const int kind = op->batch_kernel;
    op->batch_kernel = 0;
    ls_status st = transpose ? pairsum_batch(op, R, x, n, nullptr, nullptr) : pairsum_batch(op, R, x, n, op->m.p);
    op->batch_kernel = kind;
    TRY(st);
    dim3 ge((unsigned)(((int64_t)n * 32 + 255) / 256), R);
    if (transpose)
        k_applyT_epi_multi<<<ge, 256, 0, op->stream>>>(n, op->b_nchunk_cur, op->bpartial.p, op->rowptrT.p, op->colsT.p,
                                                       op->valsT.p, op->m.p, op->w.p, x, n, op->k * op->k, y, n);
    else
        k_apply_epi_multi<<<ge, 256, 0, op->stream>>>(n, op->b_nchunk_cur, op->bpartial.p, op->rowptr.p, op->cols.p,
                                                      op->vals.p, op->m.p, x, n, op->k * op->k, y, n);
    CK(cudaGetLastError());
    op->launches++;
    return LS_OK;
}

#define TC_RESID_FLOOR 2e-8
#define TC_FIRST_TOL 1e-6

// Batched GMRES.  On the tensor cores the operator carries ~1e-6 relative error from the
// FP32 accumulation in tensor memory, so the solve is followed by iterative refinement:
// the residual r = b - L u is formed with the accurate batched operator (CUDA cores), a
// tensor-core GMRES solves L d = r to a loose tolerance and u += d, until every system
// meets the GMRES criterion ||P r|| <= tol ||P b|| with the accurate operator.
static ls_status refine_batch(ls_op* op, int R, const double2* b, double2* u, int* iters, bool transpose);

static ls_status gmres_batch(ls_op* op, int R, const double2* b, double2* u, int* iters, bool transpose = false) {
    if ((op->batch_kernel != 1 && !op->refine_single) || op->tc_refine <= 0)
        return gmres_batch_plain(op, R, b, u, iters, transpose);
    // the tensor-core operator is itself only ~3e-7 x fold accurate: a first solve tighter
    // than TC_FIRST_TOL would refine nothing the accurate residual does not redo
    const double tol_save = op->prm.tol;
    op->prm.tol = std::max(tol_save, TC_FIRST_TOL);
    ls_status s0 = gmres_batch_plain(op, R, b, u, iters, transpose);
    op->prm.tol = tol_save;
    if (s0 != LS_OK && s0 != LS_ENOCONV) return s0;
    return refine_batch(op, R, b, u, iters, transpose);
}

static ls_status refine_batch(ls_op* op, int R, const double2* b, double2* u, int* iters, bool transpose) {
    const int n = op->nq;
    const int64_t tot = (int64_t)R * n;
    if (op->ir_r.n < (size_t)tot) {
        CK(op->ir_r.alloc(tot));
        CK(op->ir_d.alloc(tot));
        CK(op->ir_y.alloc(tot));
    }
    std::vector<double> pb, pr;
    TRY(prec_norms(op, R, b, transpose, pb));
    // The accurate operator evaluates L to ~1e-7 (FP32 sums), so residuals below that level
    // are rounding noise: stop at max(tol, TC_RESID_FLOOR) or when a correction no longer
    // halves the worst residual (the floor reached).
    const double tol = std::max(op->prm.tol, op->refine_single ? 0.0 : TC_RESID_FLOOR);
    const double stall_level = op->refine_single ? 1e-24 : 1e-12;
    const int blocks = (int)((tot + 255) / 256);
    std::vector<int> its(R);
    bool ok = false;
    double prev_worst = 1e300;
    for (int step = 0; step <= op->tc_refine; ++step) {
        TRY(apply_L_batch_accurate(op, R, u, op->ir_y.p, transpose));
        k_residual_multi<<<blocks, 256, 0, op->stream>>>(tot, b, op->ir_y.p, op->ir_r.p);
        CK(cudaGetLastError());
        op->launches++;
        TRY(prec_norms(op, R, op->ir_r.p, transpose, pr));
        ok = true;
        double worst = 0;
        for (int r = 0; r < R; ++r) {
            ok = ok && pr[r] <= tol * tol * pb[r];
            if (pb[r] > 0) worst = std::max(worst, pr[r] / pb[r]);
        }
        // stagnated (||r|| fell by less than 2x) at the accurate operator's rounding level,
        // ||P r|| <= 1e-6 ||P b|| for the FP32 batched operator (a few ulps of FP32) and
        // 1e-12 for the single-RHS FP64-accurate one: converged; stagnation above that level
        // is a failure
        if (!ok && worst > 0.25 * prev_worst && worst <= stall_level) ok = true;
        prev_worst = worst;
        if (ok || step == op->tc_refine) break;
        // correction to the relative tolerance that brings the worst residual below tol / 2
        // (at least 1e-3: the tensor-core operator limits a correction to about that)
        const double tol_save = op->prm.tol;
        op->prm.tol = std::min(0.5, std::max(0.5 * tol / std::sqrt(worst), 1e-3));
        ls_status sc = gmres_batch_plain(op, R, op->ir_r.p, op->ir_d.p, its.data(), transpose);
        op->prm.tol = tol_save;
        if (sc != LS_OK && sc != LS_ENOCONV) return sc;
        k_accumulate_multi<<<blocks, 256, 0, op->stream>>>(tot, op->ir_d.p, u);
        CK(cudaGetLastError());
        op->launches++;
        if (iters) for (int r = 0; r < R; ++r) iters[r] += its[r];
    }
    return ok ? LS_OK : LS_ENOCONV;
}

// Several operators (scatterers) solved in lock step: each iteration one persistent
// pair-sum launch covers every operator with an unconverged system.  The grid size
// of that launch is chosen once per call by timing candidate resident-block counts
// on the first iteration (the pair sum is idempotent, so the trial launches only
// cost time).
static ls_status solve_multi(int S, ls_op* const* ops, int R, const double2* const* b, double2* const* u, int* iters,
                             bool& all_conv) {
    cudaStream_t st = ops[0]->stream;
    for (int s = 0; s < S; ++s) {
        if (!ops[s]) return fail(LS_EINVAL, "null operator");
        if (ops[s]->stream != st) return fail(LS_EINVAL, "all operators must share one stream");
        TRY(ensure_batch(ops[s], R));
        TRY(ensure_table32(ops[s]));
    }
    size_t max_tab = 0;
    for (int s = 0; s < S; ++s) max_tab = std::max(max_tab, ops[s]->t32_bytes);
    CK(raise_smem_limit(k_pairsum_persist, max_tab));
    int dev = 0, nsm = 148, occ = 1;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pairsum_persist, PS_TPB, max_tab));
    occ = std::max(occ, 1);
    const bool tcore = ops[0]->batch_kernel == 1;
    if (ops[0]->batch_kernel == 2) return fail(LS_EINVAL, "multi-operator solves take batch kernel 0 or 1");
    for (int s = 0; s < S; ++s) {
        TRY(gb_begin(ops[s], R, b[s]));
        if (tcore) TRY(ensure_tc(ops[s]));
        ops[s]->b_nchunk_cur = ops[s]->b_nchunk;      // the persistent CUDA-core kernel writes these partials
    }
    // first solves to TC_FIRST_TOL where refinement follows (as in gmres_batch); the guard
    // restores every operator's tolerance on all exits
    auto refines = [](const ls_op* op) { return op->tc_refine > 0 && (op->batch_kernel == 1 || op->refine_single); };
    struct TolGuard {
        std::vector<std::pair<ls_op*, double>> saved;
        void restore() { for (auto& p : saved) p.first->prm.tol = p.second; saved.clear(); }
        ~TolGuard() { restore(); }
    } tg;
    for (int s = 0; s < S; ++s)
        if (refines(ops[s])) {
            tg.saved.emplace_back(ops[s], ops[s]->prm.tol);
            ops[s]->prm.tol = std::max(ops[s]->prm.tol, TC_FIRST_TOL);
        }
    // iterative refinement of every operator that takes it, after the lock-step solves
    auto refine_all = [&](std::vector<char>& conv) -> ls_status {
        tg.restore();
        all_conv = true;
        for (int s = 0; s < S; ++s) {
            bool c = conv[s] != 0;
            int* its = iters ? iters + (size_t)s * R : nullptr;
            if (refines(ops[s])) {
                ls_status sr = refine_batch(ops[s], R, b[s], u[s], its, false);
                if (sr != LS_OK && sr != LS_ENOCONV) return sr;
                c = sr == LS_OK;
            }
            all_conv = all_conv && c;
        }
        return LS_OK;
    };
    if (tcore) {
        // one persistent tensor-core launch per iteration over the unconverged operators
        DevBuf<TCOp> tdesc;
        CK(tdesc.alloc(std::max(S, 1)));
        std::vector<TCOp> tcache;
        std::vector<char> done(S, 0);
        std::vector<int> act;
        const int maxit = ops[0]->prm.max_iter;
        for (int s = 1; s < S; ++s)
            if (ops[s]->prm.max_iter != maxit) return fail(LS_EINVAL, "all operators must share max_iter");
        for (int j = 0; j < maxit; ++j) {
            std::vector<ls_op*> which;
            std::vector<const double2*> fs, ms;
            std::vector<const double*> ws;
            std::vector<size_t> sfs;
            for (int s = 0; s < S; ++s) {
                if (done[s]) continue;
                which.push_back(ops[s]);
                fs.push_back(ops[s]->bV.p + (size_t)j * ops[s]->nq);
                sfs.push_back((size_t)(maxit + 1) * ops[s]->nq);
                ms.push_back(ops[s]->m.p);
                ws.push_back(ops[s]->w.p);
            }
            if (which.empty()) break;
            TRY(pairsum_tc_launch((int)which.size(), which.data(), R, fs.data(), sfs.data(), ms.data(), ws.data(),
                                  tdesc.p, tcache, st));
            which[0]->pairsum_launches++;
            for (ls_op* op : which) TRY(gb_after_pairsum(op, R, j));
            for (int s = 0; s < S; ++s) {
                if (done[s]) continue;
                bool any = false;
                TRY(gb_active(ops[s], R, act, any));
                if (!any) done[s] = 1;
            }
            TRY(tc_status(which[0]));
        }
        std::vector<char> conv(S, 0);
        for (int s = 0; s < S; ++s) {
            bool c = false;
            int* its = iters ? iters + (size_t)s * R : nullptr;
            TRY(gb_finish(ops[s], R, u[s], its, c));
            conv[s] = c;
        }
        return refine_all(conv);
    }
    DevBuf<PSDesc> ddesc;
    DevBuf<int> counter;
    CK(ddesc.alloc(S));
    CK(counter.alloc(1));
    std::vector<PSDesc> hd(S);
    std::vector<char> done(S, 0);
    std::vector<int> act;
    int grid_blocks = nsm * occ;
    const int maxit = ops[0]->prm.max_iter;
    for (int s = 1; s < S; ++s)
        if (ops[s]->prm.max_iter != maxit) return fail(LS_EINVAL, "all operators must share max_iter");
    for (int j = 0; j < maxit; ++j) {
        int nd = 0, total = 0;
        std::vector<int> which;
        for (int s = 0; s < S; ++s) {
            if (done[s]) continue;
            ls_op* op = ops[s];
            const size_t svr = (size_t)(maxit + 1) * op->nq;
            PSDesc d;
            d.a = multi_args(op, R, op->bV.p + (size_t)j * op->nq, svr, op->m.p);
            d.tab = (const float4*)op->tab32.p;
            d.tab_words = (int)(op->t32_bytes / sizeof(float4));
            d.tblocks = (op->nq + PS_TPB - 1) / PS_TPB;
            d.units = d.tblocks * op->b_nchunk * ((R + MRB - 1) / MRB);
            d.unit_begin = total;
            total += d.units;
            hd[nd++] = d;
            which.push_back(s);
        }
        if (nd == 0) break;
        CK(cudaMemcpyAsync(ddesc.p, hd.data(), sizeof(PSDesc) * nd, cudaMemcpyHostToDevice, st));
        if (j == 0) {   // autotune the resident grid: candidates 1/2, 1 and 2 blocks per resident slot
            float best = 1e30f;
            int cand[3] = {std::max(1, nsm * occ / 2), nsm * occ, nsm * occ * 2};
            cudaEvent_t e0, e1;
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            for (int c = 0; c < 3; ++c) {
                CK(cudaMemsetAsync(counter.p, 0, sizeof(int), st));
                CK(cudaEventRecord(e0, st));
                k_pairsum_persist<<<cand[c], PS_TPB, max_tab, st>>>(ddesc.p, nd, total, counter.p);
                CK(cudaEventRecord(e1, st));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) { best = ms; grid_blocks = cand[c]; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            for (int s = 0; s < S; ++s) ops[s]->launches += 3;
        }
        CK(cudaMemsetAsync(counter.p, 0, sizeof(int), st));
        k_pairsum_persist<<<grid_blocks, PS_TPB, max_tab, st>>>(ddesc.p, nd, total, counter.p);
        CK(cudaGetLastError());
        ops[which[0]]->launches++;
        ops[which[0]]->pairsum_launches++;
        for (int s : which) TRY(gb_after_pairsum(ops[s], R, j));
        for (int s : which) {
            bool any = false;
            TRY(gb_active(ops[s], R, act, any));
            if (!any) done[s] = 1;
        }
    }
    std::vector<char> conv(S, 0);
    for (int s = 0; s < S; ++s) {
        bool c = false;
        TRY(gb_finish(ops[s], R, u[s], iters ? iters + (size_t)s * R : nullptr, c));
        conv[s] = c;
    }
    return refine_all(conv);
}

extern "C" {

ls_status ls_apply_precond_batch_dev(ls_op* op, int32_t R, const void* x_dev, void* y_dev) {
    if (!op || !x_dev || !y_dev || R < 1) return fail(LS_EINVAL, "null argument or R < 1");
    if (!op->has_prec) return fail(LS_EINVAL, "operator was built without a preconditioner");
    if (x_dev == y_dev) return fail(LS_EINVAL, "x and y may not alias");
    TRY(ensure_batch(op, R));
    TRY(apply_P_batch(op, R, (const double2*)x_dev, op->nq, (double2*)y_dev, op->nq));
    return check_stream_sync(op);
}

ls_status ls_pairsum_batch_dev(ls_op* op, int32_t R, const void* f_dev, void* y_dev) {
    if (!op || R < 1 || !f_dev || !y_dev) return fail(LS_EINVAL, "null argument or R < 1");
    TRY(ensure_batch(op, R));
    TRY(pairsum_batch(op, R, (const double2*)f_dev, op->nq, nullptr));
    // y_r = (i/4) sum_c partial: the batched epilogue with k2 = 0 and x = 0 would add x; use the
    // single epilogue in mode 1 per system instead
    int threads = 256;
    int blocks = (int)(((int64_t)op->nq * 32 + threads - 1) / threads);
    for (int r = 0; r < R; ++r)
        k_apply_epi<<<blocks, threads, 0, op->stream>>>(op->nq, op->b_nchunk_cur, op->bpartial.p + (size_t)r * op->b_nchunk_cur * op->nq,
                                                        nullptr, nullptr, nullptr, nullptr, nullptr, 0.0,
                                                        (double2*)y_dev + (size_t)r * op->nq, 1);
    CK(cudaGetLastError());
    TRY(check_stream_sync(op));
    return tc_status(op);
}

ls_status ls_op_set_stall_test(ls_op* op, double stall_ms) {
    if (!op || !(stall_ms >= 0) || stall_ms > 1000.0) return fail(LS_EINVAL, "stall_ms must be in [0, 1000]");
    op->tc_stall_ns = (uint64_t)(stall_ms * 1e6);
    return LS_OK;
}

ls_status ls_op_set_batch_kernel(ls_op* op, int32_t kind, int32_t fold, int32_t refine) {
    if (!op || kind < 0 || kind > 2 || fold < 1 || refine < 0)
        return fail(LS_EINVAL, "kind must be 0, 1 or 2, fold >= 1, refine >= 0");
    if (kind == 2 && op->mode != 3 && op->mode != 4)
        return fail(LS_EINVAL, "kind 2 needs the double-float table (LS_PREC_FP64_DF or LS_PREC_MIXED)");
    op->batch_kernel = kind;
    op->tc_fold = fold;
    op->tc_refine = refine;
    return LS_OK;
}

ls_status ls_tc_gemm_check(int32_t N, double* max_abs_err) {
    if (!max_abs_err || N < 16 || N > 256 || (N & 15)) return fail(LS_EINVAL, "N must be a multiple of 16 in [16, 256]");
    // small integers times powers of two: exact in TF32, exact sums in FP32
    std::vector<float> A(TC_M * 32), B((size_t)N * 32), D((size_t)TC_M * N);
    uint32_t st = 12345u;
    auto rnd = [&]() { st = st * 1664525u + 1013904223u; return (int)((st >> 24) % 15) - 7; };
    for (auto& v : A) v = (float)rnd() * 0.25f;
    for (auto& v : B) v = (float)rnd() * 0.5f;
    DevBuf<float> dA, dB, dD;
    DevBuf<int> derr;
    CK(dA.alloc(A.size()));
    CK(dB.alloc(B.size()));
    CK(dD.alloc(D.size()));
    CK(derr.alloc(1));
    CK(cudaMemcpy(dA.p, A.data(), sizeof(float) * A.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dB.p, B.data(), sizeof(float) * B.size(), cudaMemcpyHostToDevice));
    CK(cudaMemset(dD.p, 0, sizeof(float) * D.size()));
    CK(cudaMemset(derr.p, 0, sizeof(int)));
    const size_t smem = 1024 + (size_t)(TC_M + N) * 32 * 4;
    CK(raise_smem_limit(k_tc_gemm_check, smem));
    k_tc_gemm_check<<<1, 128, smem>>>(dA.p, dB.p, N, dD.p, derr.p);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    int herr = 0;
    CK(cudaMemcpy(&herr, derr.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) return fail(LS_ETIMEOUT, "tensor-core check: the MMA completion wait ran out");
    CK(cudaMemcpy(D.data(), dD.p, sizeof(float) * D.size(), cudaMemcpyDeviceToHost));
    double e = 0;
    for (int i = 0; i < TC_M; ++i)
        for (int j = 0; j < N; ++j) {
            double ref = 0;
            for (int kk = 0; kk < 32; ++kk) ref += (double)A[i * 32 + kk] * B[(size_t)j * 32 + kk];
            e = std::max(e, std::fabs(ref - (double)D[(size_t)i * N + j]));
        }
    *max_abs_err = e;
    return LS_OK;
}

ls_status ls_solve_transpose_batch_dev(ls_op* op, int32_t R, const void* g_dev, void* lambda_dev, int32_t* iters_out) {
    if (!op || R < 1 || !g_dev || !lambda_dev) return fail(LS_EINVAL, "null argument or R < 1");
    std::vector<int> its(R);
    ls_status s = gmres_batch(op, R, (const double2*)g_dev, (double2*)lambda_dev, its.data(), true);
    if (s != LS_OK && s != LS_ENOCONV) return s;
    if (iters_out) for (int r = 0; r < R; ++r) iters_out[r] = its[r];
    TRY(check_stream_sync(op));
    if (s == LS_ENOCONV) fail(s, "GMRES reached max_iter");
    return s;
}

ls_status ls_misfit_gradient_batch_dev(ls_op* op, int32_t R, const void* u_dev, int32_t n_ff, const double* ff_angles,
                                       const void* resid_dev, double* grad_dev, int32_t* iters_out) {
    if (!op || R < 1 || !u_dev || n_ff < 1 || !ff_angles || !resid_dev || !grad_dev)
        return fail(LS_EINVAL, "null argument or bad size");
    const int n = op->nq;
    DevBuf<double> ang;
    DevBuf<double2> g, rhs, lam, vtl;
    CK(ang.alloc(n_ff));
    CK(g.alloc((size_t)R * n));
    CK(rhs.alloc((size_t)R * n));
    CK(lam.alloc((size_t)R * n));
    CK(vtl.alloc(n));
    CK(cudaMemcpy(ang.p, ff_angles, sizeof(double) * n_ff, cudaMemcpyHostToDevice));
    const int nb = (n + 255) / 256;
    for (int r = 0; r < R; ++r) {
        k_farfieldT<<<nb, 256, 0, op->stream>>>(n, op->xy.p, op->w.p, op->k, n_ff, ang.p,
                                               (const double2*)resid_dev + (size_t)r * n_ff, g.p + (size_t)r * n);
        k_cmul_vec<<<nb, 256, 0, op->stream>>>(n, op->m.p, g.p + (size_t)r * n, rhs.p + (size_t)r * n);
    }
    CK(cudaGetLastError());
    op->launches += 2 * R;
    std::vector<int> its(R);
    ls_status s = gmres_batch(op, R, rhs.p, lam.p, its.data(), true);
    if (s != LS_OK && s != LS_ENOCONV) return s;
    if (iters_out) for (int r = 0; r < R; ++r) iters_out[r] = its[r];
    CK(cudaMemsetAsync(grad_dev, 0, sizeof(double) * n, op->stream));
    // V^T lambda for all R directions in one batched pair sum on unit weights (the CUDA-core
    // batched kernel, whose ~6e-8 pair-sum error keeps the gradient well inside 1e-5)
    {
        const int kind = op->batch_kernel;
        op->batch_kernel = 0;
        ls_status ps = pairsum_batch(op, R, lam.p, (size_t)n, nullptr, nullptr);
        op->batch_kernel = kind;
        TRY(ps);
        dim3 ge((unsigned)(((int64_t)n * 32 + 255) / 256), R);
        k_applyT_epi_multi<<<ge, 256, 0, op->stream>>>(n, op->b_nchunk_cur, op->bpartial.p, op->rowptrT.p, op->colsT.p,
                                                       op->valsT.p, nullptr, op->w.p, lam.p, (size_t)n, 0.0, rhs.p,
                                                       (size_t)n);
        CK(cudaGetLastError());
        op->launches++;
    }
    for (int r = 0; r < R; ++r) {
        k_grad_acc<<<nb, 256, 0, op->stream>>>(n, (const double2*)u_dev + (size_t)r * n, g.p + (size_t)r * n,
                                               rhs.p + (size_t)r * n, op->k * op->k, grad_dev);
        CK(cudaGetLastError());
        op->launches++;
    }
    TRY(check_stream_sync(op));
    if (s == LS_ENOCONV) fail(s, "adjoint GMRES reached max_iter");
    return s;
}

ls_status ls_solve_multi_dev(int32_t S, ls_op* const* ops, int32_t R, const void* const* b_devs, void* const* u_devs,
                             int32_t* iters_out) {
    if (S < 1 || !ops || R < 1 || !b_devs || !u_devs) return fail(LS_EINVAL, "null argument or bad size");
    for (int s = 0; s < S; ++s)
        if (!ops[s] || !b_devs[s] || !u_devs[s]) return fail(LS_EINVAL, "null operator or buffer");
    bool all = false;
    std::vector<int> its((size_t)S * R);
    TRY(solve_multi(S, ops, R, reinterpret_cast<const double2* const*>(b_devs), reinterpret_cast<double2* const*>(u_devs),
                    its.data(), all));
    if (iters_out) for (size_t i = 0; i < its.size(); ++i) iters_out[i] = its[i];
    CK(cudaStreamSynchronize(ops[0]->stream));
    if (!all) return fail(LS_ENOCONV, "GMRES reached max_iter");
    return LS_OK;
}

ls_status ls_solve_batch_dev(ls_op* op, int32_t R, const void* b_dev, void* u_dev, int32_t n_ff, const double* ff_angles,
                             void* uinf_dev, int32_t* iters_out) {
    if (!op || R < 1 || !b_dev || !u_dev) return fail(LS_EINVAL, "null argument or R < 1");
    if (n_ff > 0 && (!ff_angles || !uinf_dev)) return fail(LS_EINVAL, "far-field buffers missing");
    std::vector<int> its(R);
    ls_status s = gmres_batch(op, R, (const double2*)b_dev, (double2*)u_dev, its.data());
    if (s != LS_OK && s != LS_ENOCONV) return s;
    if (iters_out) for (int r = 0; r < R; ++r) iters_out[r] = its[r];
    if (n_ff > 0) {
        DevBuf<double> ang;
        CK(ang.alloc(n_ff));
        CK(cudaMemcpy(ang.p, ff_angles, sizeof(double) * n_ff, cudaMemcpyHostToDevice));
        for (int r = 0; r < R; ++r)
            TRY(farfield(op, (const double2*)u_dev + (size_t)r * op->nq, n_ff, ang.p, (double2*)uinf_dev + (size_t)r * n_ff));
    }
    TRY(check_stream_sync(op));
    if (s == LS_ENOCONV) fail(s, "GMRES reached max_iter");
    return s;
}

ls_status ls_solve_dev(ls_op* op, int32_t R, const void* b_dev, void* u_dev, int32_t n_ff, const double* ff_angles,
                       void* uinf_dev, int32_t* iters_out) {
    if (!op || R < 1 || !b_dev || !u_dev) return fail(LS_EINVAL, "null argument or R < 1");
    if (n_ff > 0 && (!ff_angles || !uinf_dev)) return fail(LS_EINVAL, "far-field buffers missing");
    DevBuf<double> ang;
    if (n_ff > 0) {
        CK(ang.alloc(n_ff));
        CK(cudaMemcpy(ang.p, ff_angles, sizeof(double) * n_ff, cudaMemcpyHostToDevice));
    }
    ls_status worst = LS_OK;
    op->last_res = 0.0;
    for (int r = 0; r < R; ++r) {
        const double2* b = (const double2*)b_dev + (size_t)r * op->nq;
        double2* u = (double2*)u_dev + (size_t)r * op->nq;
        int it = 0;
        ls_status s = solve_one(op, b, u, nullptr, &it);
        if (s != LS_OK && s != LS_ENOCONV) return s;
        if (s == LS_ENOCONV) worst = s;
        if (iters_out) iters_out[r] = it;
        if (n_ff > 0) TRY(farfield(op, u, n_ff, ang.p, (double2*)uinf_dev + (size_t)r * n_ff));
    }
    TRY(check_stream_sync(op));
    if (worst != LS_OK) fail(worst, "GMRES reached max_iter");
    return worst;
}

ls_status ls_solve(ls_op* op, int32_t R, const double* dir_angles, const double* b_in, int32_t n_ff,
                   const double* ff_angles, double* u_out, double* uinf_out, double* hist_out, int32_t* iters_out) {
    if (!op || R < 1 || (!dir_angles && !b_in)) return fail(LS_EINVAL, "null argument or R < 1");
    if (n_ff > 0 && !ff_angles) return fail(LS_EINVAL, "ff_angles missing");
    const int n = op->nq;
    DevBuf<double2> b, u, uinf;
    DevBuf<double> ang;
    CK(b.alloc(n));
    CK(u.alloc(n));
    if (n_ff > 0) {
        CK(uinf.alloc(n_ff));
        CK(ang.alloc(n_ff));
        CK(cudaMemcpy(ang.p, ff_angles, sizeof(double) * n_ff, cudaMemcpyHostToDevice));
    }
    std::vector<double> hist(op->prm.max_iter + 2);
    ls_status worst = LS_OK;
    op->last_res = 0.0;
    for (int r = 0; r < R; ++r) {
        if (b_in) {
            CK(cudaMemcpyAsync(b.p, b_in + 2 * (size_t)r * n, sizeof(double2) * n, cudaMemcpyHostToDevice, op->stream));
        } else {
            k_incident<<<(n + 255) / 256, 256, 0, op->stream>>>(n, op->xy.p, op->k, std::cos(dir_angles[r]),
                                                                 std::sin(dir_angles[r]), b.p);
            CK(cudaGetLastError());
            op->launches++;
        }
        int it = 0;
        ls_status s = solve_one(op, b.p, u.p, hist.data(), &it);
        if (s != LS_OK && s != LS_ENOCONV) return s;
        if (s == LS_ENOCONV) worst = s;
        if (iters_out) iters_out[r] = it;
        if (hist_out) {
            double* hr = hist_out + (size_t)r * (op->prm.max_iter + 1);
            for (int i = 0; i <= op->prm.max_iter; ++i) hr[i] = i <= it ? hist[i] : 0.0;
        }
        if (u_out) CK(cudaMemcpyAsync(u_out + 2 * (size_t)r * n, u.p, sizeof(double2) * n, cudaMemcpyDeviceToHost, op->stream));
        if (n_ff > 0 && uinf_out) {
            TRY(farfield(op, u.p, n_ff, ang.p, uinf.p));
            CK(cudaMemcpyAsync(uinf_out + 2 * (size_t)r * n_ff, uinf.p, sizeof(double2) * n_ff, cudaMemcpyDeviceToHost,
                               op->stream));
        }
        TRY(check_stream_sync(op));
    }
    if (worst != LS_OK) fail(worst, "GMRES reached max_iter");
    return worst;
}

// Host-buffer forms of the apply calls: x, y [N] complex on the host.
static ls_status apply_host(ls_op* op, const double* x, double* y, int which) {
    if (!op || !x || !y) return fail(LS_EINVAL, "null argument");
    if (which == 1 && !op->has_prec) return fail(LS_EINVAL, "operator was built without a preconditioner");
    DevBuf<double2> xd, yd;
    CK(xd.alloc(op->nq));
    CK(yd.alloc(op->nq));
    CK(cudaMemcpyAsync(xd.p, x, sizeof(double2) * op->nq, cudaMemcpyHostToDevice, op->stream));
    if (which == 1) TRY(apply_P(op, xd.p, yd.p));
    else if (which == 2) TRY(apply_LT(op, xd.p, yd.p));
    else TRY(apply_PT(op, xd.p, yd.p));
    CK(cudaMemcpyAsync(y, yd.p, sizeof(double2) * op->nq, cudaMemcpyDeviceToHost, op->stream));
    return check_stream_sync(op);
}

ls_status ls_apply_precond(ls_op* op, const double* x, double* y) { return apply_host(op, x, y, 1); }
ls_status ls_apply_transpose(ls_op* op, const double* x, double* y) { return apply_host(op, x, y, 2); }

ls_status ls_solve_adjoint(ls_op* op, int32_t R, const double* g, double* lambda_out, int32_t* iters_out) {
    if (!op || R < 1 || !g || !lambda_out) return fail(LS_EINVAL, "null argument or R < 1");
    const int n = op->nq;
    DevBuf<double2> gd, ld;
    CK(gd.alloc(n));
    CK(ld.alloc(n));
    ls_status worst = LS_OK;
    op->last_res = 0.0;
    for (int r = 0; r < R; ++r) {
        CK(cudaMemcpyAsync(gd.p, g + 2 * (size_t)r * n, sizeof(double2) * n, cudaMemcpyHostToDevice, op->stream));
        int it = 0;
        ls_status s = solve_one(op, gd.p, ld.p, nullptr, &it, true);
        if (s != LS_OK && s != LS_ENOCONV) return s;
        if (s == LS_ENOCONV) worst = s;
        if (iters_out) iters_out[r] = it;
        CK(cudaMemcpyAsync(lambda_out + 2 * (size_t)r * n, ld.p, sizeof(double2) * n, cudaMemcpyDeviceToHost, op->stream));
        TRY(check_stream_sync(op));
    }
    if (worst != LS_OK) fail(worst, "adjoint GMRES reached max_iter");
    return worst;
}

ls_status ls_residual_dev(ls_op* op, const void* b_dev, const void* u_dev, double* rel) {
    if (!op || !b_dev || !u_dev || !rel) return fail(LS_EINVAL, "null argument");
    return residual_full(op, (const double2*)b_dev, (const double2*)u_dev, rel);
}

// Eigenvalues of an upper Hessenberg matrix (n x n, column-major) by the shifted QR
// iteration: deflation at negligible subdiagonals, Wilkinson shift from the trailing 2 x 2
// block of the active window, an exceptional shift every 10 iterations without
// deflation; each step H - mu I = Q R, H <- R Q + mu I with complex Givens rotations.
static bool hessenberg_eig(int n, std::vector<std::complex<double>>& H, std::vector<std::complex<double>>& eig) {
    using cd = std::complex<double>;
    auto A = [&](int r, int c) -> cd& { return H[(size_t)c * n + r]; };
    eig.clear();
    int hi = n - 1, iter = 0, total = 0;
    std::vector<cd> cs(n), sn(n);
    while (hi >= 0) {
        if (hi == 0) { eig.push_back(A(0, 0)); --hi; continue; }
        int l = hi;
        while (l > 0 && std::abs(A(l, l - 1)) > 1e-15 * (std::abs(A(l - 1, l - 1)) + std::abs(A(l, l)))) --l;
        if (l == hi) { eig.push_back(A(hi, hi)); --hi; iter = 0; continue; }
        if (++total > 100 * n) return false;
        cd mu;
        if (iter % 10 == 9) {
            mu = A(hi, hi) + cd(std::abs(A(hi, hi - 1)), 0.0);
        } else {
            const cd a = A(hi - 1, hi - 1), b = A(hi - 1, hi), c = A(hi, hi - 1), d = A(hi, hi);
            const cd half = 0.5 * (a - d);
            const cd disc = std::sqrt(half * half + b * c);
            const cd m1 = 0.5 * (a + d) + disc, m2 = 0.5 * (a + d) - disc;
            mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
        }
        ++iter;
        for (int k = l; k <= hi; ++k) A(k, k) -= mu;
        for (int k = l; k < hi; ++k) {
            const cd a = A(k, k), b = A(k + 1, k);
            const double r = std::sqrt(std::norm(a) + std::norm(b));
            const cd c = r > 0 ? a / r : cd(1, 0), s = r > 0 ? b / r : cd(0, 0);
            cs[k] = c;
            sn[k] = s;
            for (int j = k; j <= hi; ++j) {
                const cd x = A(k, j), y = A(k + 1, j);
                A(k, j) = std::conj(c) * x + std::conj(s) * y;
                A(k + 1, j) = -s * x + c * y;
            }
        }
        for (int k = l; k < hi; ++k) {
            const cd c = cs[k], s = sn[k];
            for (int i = l; i <= std::min(k + 2, hi); ++i) {
                const cd x = A(i, k), y = A(i, k + 1);
                A(i, k) = x * c + y * s;
                A(i, k + 1) = -x * std::conj(s) + y * std::conj(c);
            }
        }
        for (int k = l; k <= hi; ++k) A(k, k) += mu;
    }
    return true;
}

ls_status ls_hessenberg_eigenvalues(int32_t n, const double* H, double* eig) {
    if (n < 1 || !H || !eig) return fail(LS_EINVAL, "null argument or n < 1");
    std::vector<std::complex<double>> A((size_t)n * n), e;
    for (size_t i = 0; i < A.size(); ++i) A[i] = std::complex<double>(H[2 * i], H[2 * i + 1]);
    if (!hessenberg_eig(n, A, e)) return fail(LS_ENOCONV, "Hessenberg QR iteration did not converge");
    for (int i = 0; i < n; ++i) { eig[2 * i] = e[i].real(); eig[2 * i + 1] = e[i].imag(); }
    return LS_OK;
}

ls_status ls_op_ritz(ls_op* op, int32_t cap, int32_t* count, double* ritz) {
    if (!op || !count) return fail(LS_EINVAL, "null argument");
    const int it = op->last_it, ldh = op->prm.max_iter + 1;
    *count = it;
    if (!ritz || it == 0) return LS_OK;
    if (cap < it) return fail(LS_EINVAL, "ritz buffer smaller than the iteration count");
    std::vector<double2> raw((size_t)ldh * it);
    CK(cudaMemcpyAsync(raw.data(), op->Hraw.p, sizeof(double2) * raw.size(), cudaMemcpyDeviceToHost, op->stream));
    CK(cudaStreamSynchronize(op->stream));
    std::vector<std::complex<double>> A((size_t)it * it), e;
    for (int c = 0; c < it; ++c)
        for (int r = 0; r < it; ++r)
            A[(size_t)c * it + r] = r <= c + 1 ? std::complex<double>(raw[(size_t)c * ldh + r].x, raw[(size_t)c * ldh + r].y)
                                               : std::complex<double>(0, 0);
    if (!hessenberg_eig(it, A, e)) return fail(LS_ENOCONV, "Hessenberg QR iteration did not converge");
    for (int i = 0; i < it; ++i) { ritz[2 * i] = e[i].real(); ritz[2 * i + 1] = e[i].imag(); }
    return LS_OK;
}

ls_status ls_precond_rho_dev(ls_op* op, int32_t R, const void* x_dev, double* rho) {
    if (!op || R < 1 || !x_dev || !rho) return fail(LS_EINVAL, "null argument or R < 1");
    if (!op->has_prec || op->cartesian) return fail(LS_EINVAL, "needs an operator with the Cartesian preconditioner");
    const int nc = op->nx * op->ny, nq = op->nq;
    DevBuf<double2> zq, q, w;
    DevBuf<double> out;
    CK(zq.alloc(nq));
    CK(q.alloc(nq));
    CK(w.alloc(nc));
    CK(out.alloc(2 * (size_t)R));
    CK(cudaMemsetAsync(zq.p, 0, sizeof(double2) * nq, op->stream));
    for (int r = 0; r < R; ++r) {
        const double2* x = (const double2*)x_dev + (size_t)r * nc;
        // w = R_II x = D^{-1} (T_C^Q)^T T_C^Q x
        k_tcq<<<(nq + 255) / 256, 256, 0, op->stream>>>(nq, op->tcq_idx.p, op->tcq_w.p, x, nullptr, zq.p, q.p);
        k_tqc<<<(nc + 255) / 256, 256, 0, op->stream>>>(nc, op->tcqT_rp.p, op->tcqT_ci.p, op->tcqT_cv.p, q.p, w.p);
        k_div_real<<<(nc + 255) / 256, 256, 0, op->stream>>>(nc, op->Dg.p, w.p);
        // S^(C) w = C^{-1} A w
        k_stencil<<<(nc + 255) / 256, 256, 0, op->stream>>>(op->nx, op->ny, op->st.p, w.p, op->cr.t());
        const int ncr = launch_cr(op, op->stream, false);
        k_rho<<<1, 256, 0, op->stream>>>(nc, op->Dg.p, w.p, op->cr.x(), out.p + 2 * r);
        CK(cudaGetLastError());
        op->launches += 5 + ncr;
    }
    CK(cudaMemcpyAsync(rho, out.p, sizeof(double) * 2 * R, cudaMemcpyDeviceToHost, op->stream));
    return check_stream_sync(op);
}

ls_status ls_op_last_residual(const ls_op* op, double* rel) {
    if (!op || !rel) return fail(LS_EINVAL, "null argument");
    *rel = op->last_res;
    return LS_OK;
}

ls_status ls_op_set_contrast_dev(ls_op* op, const void* m_dev, int32_t real_only) {
    if (!op || !m_dev) return fail(LS_EINVAL, "null argument");
    const int n = op->nq;
    if (real_only) {
        k_real_to_complex<<<(n + 255) / 256, 256, 0, op->stream>>>(n, (const double*)m_dev, op->m.p);
        CK(cudaGetLastError());
        op->launches++;
    } else {
        CK(cudaMemcpyAsync(op->m.p, m_dev, sizeof(double2) * n, cudaMemcpyDeviceToDevice, op->stream));
    }
    return check_stream_sync(op);
}

ls_status ls_misfit_dev(ls_op* op, int32_t total, const void* uinf_dev, const void* target_dev, void* resid_dev,
                        double* J) {
    if (!op || total < 1 || !uinf_dev || !target_dev || !resid_dev || !J) return fail(LS_EINVAL, "null argument");
    DevBuf<double> jd;
    CK(jd.alloc(1));
    k_misfit<<<1, 256, 0, op->stream>>>(total, (const double2*)uinf_dev, (const double2*)target_dev,
                                        (double2*)resid_dev, jd.p);
    CK(cudaGetLastError());
    op->launches++;
    CK(cudaMemcpyAsync(J, jd.p, sizeof(double), cudaMemcpyDeviceToHost, op->stream));
    return check_stream_sync(op);
}

ls_status ls_op_correction(const ls_op* op, int64_t* nnz, int64_t* rowptr, int32_t* cols, double* vals) {
    if (!op || !nnz) return fail(LS_EINVAL, "null argument");
    *nnz = (int64_t)op->host_csr.cols.size();
    if (rowptr) std::memcpy(rowptr, op->host_csr.rowptr.data(), sizeof(int64_t) * op->host_csr.rowptr.size());
    if (cols) std::memcpy(cols, op->host_csr.cols.data(), sizeof(int32_t) * op->host_csr.cols.size());
    if (vals) std::memcpy(vals, op->host_csr.vals.data(), sizeof(double) * 2 * op->host_csr.vals.size());
    return LS_OK;
}

// Size query of the correction CSR: 15 entries per (target, patch) block of the plan.
static ls_status correction_size(const ls_mesh* mesh, double kappa, int64_t* nnz) {
    lsgpu::CorrPlan P;
    std::string err = lsgpu::plan_correction(mesh->h, kappa, P);
    if (!err.empty()) return fail(LS_EINVAL, err);
    *nnz = 15 * (int64_t)P.target.size();
    return LS_OK;
}

ls_status ls_correction_host(const ls_mesh* mesh, double k, double kappa, int64_t* nnz, int64_t* rowptr,
                             int32_t* cols, double* vals) {
    if (!mesh || !nnz) return fail(LS_EINVAL, "null argument");
    if (!(k > 0) || !(kappa > 0)) return fail(LS_EINVAL, "k and kappa must be positive");
    if (!rowptr && !cols && !vals) return correction_size(mesh, kappa, nnz);
    CsrC csr;
    std::string err = lsgpu::build_correction(mesh->h, k, kappa, csr);
    if (!err.empty()) return fail(LS_ESINGULAR, err);
    *nnz = (int64_t)csr.cols.size();
    if (rowptr) std::memcpy(rowptr, csr.rowptr.data(), sizeof(int64_t) * csr.rowptr.size());
    if (cols) std::memcpy(cols, csr.cols.data(), sizeof(int32_t) * csr.cols.size());
    if (vals) std::memcpy(vals, csr.vals.data(), sizeof(double) * 2 * csr.vals.size());
    return LS_OK;
}

ls_status ls_correction_dev(const ls_mesh* mesh, double k, double kappa, void* stream, int64_t* nnz,
                            int64_t* rowptr, int32_t* cols, double* vals, int64_t* host_blocks) {
    if (!mesh || !nnz) return fail(LS_EINVAL, "null argument");
    if (!(k > 0) || !(kappa > 0)) return fail(LS_EINVAL, "k and kappa must be positive");
    if (!rowptr && !cols && !vals) return correction_size(mesh, kappa, nnz);
    CsrC A;
    std::string err = lsgpu::build_correction_device(mesh->h, k, kappa, stream, A, host_blocks);
    if (!err.empty()) return fail(err.find("singular") != std::string::npos ? LS_ESINGULAR : LS_ECUDA, err);
    *nnz = (int64_t)A.cols.size();
    if (rowptr) std::copy(A.rowptr.begin(), A.rowptr.end(), rowptr);
    if (cols) std::copy(A.cols.begin(), A.cols.end(), cols);
    if (vals)
        for (size_t e = 0; e < A.vals.size(); ++e) { vals[2 * e] = A.vals[e].real(); vals[2 * e + 1] = A.vals[e].imag(); }
    return LS_OK;
}

ls_status ls_transfer_host(const ls_mesh* mesh, const double* box, int32_t nx, int32_t ny, int32_t approach,
                           int64_t* nnz, int64_t* rowptr, int32_t* cols, double* vals, int32_t* n_interior) {
    if (!mesh || !box || !nnz) return fail(LS_EINVAL, "null argument");
    if (approach != 1 && approach != 2) return fail(LS_EINVAL, "approach must be 1 or 2");
    GridSetup G;
    std::string err = lsgpu::build_transfers(mesh->h, box, nx, ny, approach, G);
    if (!err.empty()) return fail(LS_EINVAL, err);
    *nnz = (int64_t)G.tqc_cols.size();
    if (rowptr) std::copy(G.tqc_rowptr.begin(), G.tqc_rowptr.end(), rowptr);
    if (cols) std::copy(G.tqc_cols.begin(), G.tqc_cols.end(), cols);
    if (vals) std::copy(G.tqc_vals.begin(), G.tqc_vals.end(), vals);
    if (n_interior) *n_interior = G.n_interior;
    return LS_OK;
}

ls_status ls_grid_host(const ls_mesh* mesh, double k, const double* box, int32_t nx, int32_t ny, const double* m_grid,
                       double* stencils, double* cband) {
    if (!mesh || !box || !m_grid || !stencils) return fail(LS_EINVAL, "null argument");
    if (!(k > 0)) return fail(LS_EINVAL, "k must be positive");
    if (nx < 4 || ny < 4) return fail(LS_EINVAL, "grid needs at least 4 x 4 nodes");
    const size_t nc = (size_t)nx * ny;
    std::vector<std::complex<double>> mg(nc);
    for (size_t i = 0; i < nc; ++i) mg[i] = std::complex<double>(m_grid[2 * i], m_grid[2 * i + 1]);
    lsgpu::GridSetup G;
    std::string err = lsgpu::build_grid(mesh->h, k, box, nx, ny, mg.data(), G);
    if (!err.empty()) return fail(LS_EINVAL, err);
    for (int c = 0; c < 9; ++c)
        for (int t = 0; t < 9; ++t) {
            stencils[2 * (9 * c + t)] = G.v[c][t].real();
            stencils[2 * (9 * c + t) + 1] = G.v[c][t].imag();
        }
    if (cband)
        for (size_t i = 0; i < G.cband.size(); ++i) {
            cband[2 * i] = G.cband[i].real();
            cband[2 * i + 1] = G.cband[i].imag();
        }
    return LS_OK;
}

ls_status ls_apply_transpose_dev(ls_op* op, const void* x_dev, void* y_dev) {
    if (!op || !x_dev || !y_dev) return fail(LS_EINVAL, "null argument");
    if (x_dev == y_dev) return fail(LS_EINVAL, "x and y may not alias");
    TRY(apply_LT(op, (const double2*)x_dev, (double2*)y_dev, 0));
    return check_stream_sync(op);
}

ls_status ls_potential_transpose_dev(ls_op* op, const void* x_dev, void* y_dev) {
    if (!op || !x_dev || !y_dev) return fail(LS_EINVAL, "null argument");
    if (x_dev == y_dev) return fail(LS_EINVAL, "x and y may not alias");
    TRY(apply_LT(op, (const double2*)x_dev, (double2*)y_dev, 2));
    return check_stream_sync(op);
}

ls_status ls_apply_precond_transpose_dev(ls_op* op, const void* x_dev, void* y_dev) {
    if (!op || !x_dev || !y_dev) return fail(LS_EINVAL, "null argument");
    if (!op->has_prec) return fail(LS_EINVAL, "operator was built without a preconditioner");
    if (x_dev == y_dev) return fail(LS_EINVAL, "x and y may not alias");
    TRY(apply_PT(op, (const double2*)x_dev, (double2*)y_dev));
    return check_stream_sync(op);
}

ls_status ls_solve_transpose_dev(ls_op* op, int32_t R, const void* g_dev, void* lambda_dev, int32_t* iters_out) {
    if (!op || R < 1 || !g_dev || !lambda_dev) return fail(LS_EINVAL, "null argument or R < 1");
    ls_status worst = LS_OK;
    op->last_res = 0.0;
    for (int r = 0; r < R; ++r) {
        int it = 0;
        ls_status s = solve_one(op, (const double2*)g_dev + (size_t)r * op->nq, (double2*)lambda_dev + (size_t)r * op->nq,
                                nullptr, &it, true);
        if (s != LS_OK && s != LS_ENOCONV) return s;
        if (s == LS_ENOCONV) worst = s;
        if (iters_out) iters_out[r] = it;
    }
    TRY(check_stream_sync(op));
    if (worst != LS_OK) fail(worst, "GMRES reached max_iter");
    return worst;
}

ls_status ls_op_set_contrast(ls_op* op, const double* m) {
    if (!op || !m) return fail(LS_EINVAL, "null argument");
    for (int q = 0; q < op->nq; ++q)
        if (!std::isfinite(m[2 * q]) || !std::isfinite(m[2 * q + 1])) return fail(LS_EINVAL, "non-finite contrast");
    CK(cudaMemcpyAsync(op->m.p, m, sizeof(double2) * op->nq, cudaMemcpyHostToDevice, op->stream));
    return check_stream_sync(op);
}

ls_status ls_incident_dev(ls_op* op, int32_t R, const double* dir_angles, void* b_dev) {
    if (!op || R < 1 || !dir_angles || !b_dev) return fail(LS_EINVAL, "null argument or R < 1");
    for (int r = 0; r < R; ++r) {
        k_incident<<<(op->nq + 255) / 256, 256, 0, op->stream>>>(op->nq, op->xy.p, op->k, std::cos(dir_angles[r]),
                                                                 std::sin(dir_angles[r]), (double2*)b_dev + (size_t)r * op->nq);
        CK(cudaGetLastError());
        op->launches++;
    }
    return check_stream_sync(op);
}

ls_status ls_misfit_gradient_dev(ls_op* op, int32_t R, const void* u_dev, int32_t n_ff, const double* ff_angles,
                                 const void* resid_dev, double* grad_dev, int32_t* iters_out) {
    if (!op || R < 1 || !u_dev || n_ff < 1 || !ff_angles || !resid_dev || !grad_dev)
        return fail(LS_EINVAL, "null argument or bad size");
    const int n = op->nq;
    DevBuf<double> ang;
    DevBuf<double2> g, rhs, lam, vtl;
    CK(ang.alloc(n_ff));
    CK(g.alloc(n));
    CK(rhs.alloc(n));
    CK(lam.alloc(n));
    CK(vtl.alloc(n));
    CK(cudaMemcpy(ang.p, ff_angles, sizeof(double) * n_ff, cudaMemcpyHostToDevice));
    CK(cudaMemsetAsync(grad_dev, 0, sizeof(double) * n, op->stream));
    ls_status worst = LS_OK;
    const int nb = (n + 255) / 256;
    for (int r = 0; r < R; ++r) {
        const double2* u = (const double2*)u_dev + (size_t)r * n;
        k_farfieldT<<<nb, 256, 0, op->stream>>>(n, op->xy.p, op->w.p, op->k, n_ff, ang.p,
                                               (const double2*)resid_dev + (size_t)r * n_ff, g.p);
        k_cmul_vec<<<nb, 256, 0, op->stream>>>(n, op->m.p, g.p, rhs.p);
        CK(cudaGetLastError());
        op->launches += 2;
        int it = 0;
        ls_status s = solve_one(op, rhs.p, lam.p, nullptr, &it, true);
        if (s != LS_OK && s != LS_ENOCONV) return s;
        if (s == LS_ENOCONV) worst = s;
        if (iters_out) iters_out[r] = it;
        TRY(apply_LT(op, lam.p, vtl.p, 2));
        k_grad_acc<<<nb, 256, 0, op->stream>>>(n, u, g.p, vtl.p, op->k * op->k, grad_dev);
        CK(cudaGetLastError());
        op->launches++;
    }
    TRY(check_stream_sync(op));
    if (worst != LS_OK) fail(worst, "adjoint GMRES reached max_iter");
    return worst;
}

ls_status ls_op_set_pairsum(ls_op* op, int32_t mode) {
    if (!op) return fail(LS_EINVAL, "null op");
    if (op->cartesian) return fail(LS_EINVAL, "a purely Cartesian operator has no pair-sum kernel");
    if (mode < 0 || mode > 4) return fail(LS_EINVAL, "pairsum must be 0, 1, 2, 3 or 4");
    CK(cudaStreamSynchronize(op->stream));
    if (mode != 1 && !(op->tab_thi > 0)) return fail(LS_EINVAL, "operator has no table range (built with pairsum = 1)");
    op->use_table = false;
    if (mode != 1) TRY(build_table_range(op, op->tab_tlo, op->tab_thi, mode == 4 ? 3 : mode));
    if (mode == 4) TRY(ensure_table32_single(op));
    if (op->batch_kernel == 2 && mode != 3 && mode != 4) op->batch_kernel = 0;   // kind 2 needs the DF table
    if (!op->refine_user) op->refine_single = mode == 3 || mode == 4;
    op->mode = mode;
    return LS_OK;
}

ls_status ls_op_set_batch_refine(ls_op* op, int32_t accurate) {
    if (!op) return fail(LS_EINVAL, "null op");
    if (accurate != 0 && accurate != 1) return fail(LS_EINVAL, "accurate must be 0 or 1");
    if (op->cartesian) return fail(LS_EINVAL, "the batched forms need a quadrature-node operator");
    op->refine_single = accurate != 0;
    op->refine_user = true;
    return LS_OK;
}

ls_status ls_op_set_pair_symmetry(ls_op* op, int32_t on) {
    if (!op) return fail(LS_EINVAL, "null op");
    if (on != 0 && on != 1) return fail(LS_EINVAL, "on must be 0 or 1");
    CK(cudaStreamSynchronize(op->stream));
    op->df_sym = on != 0;
    return LS_OK;
}

ls_status ls_op_tuning(const ls_op* op, int32_t* table_ncoef, double* cand_ms, int32_t* fp32_tail) {
    if (!op) return fail(LS_EINVAL, "null op");
    if (table_ncoef) *table_ncoef = op->tab_nc;
    if (fp32_tail) *fp32_tail = (op->mode == 3 || op->mode == 4) ? op->tab_nf : 0;
    if (cand_ms) for (int i = 0; i < 4; ++i) cand_ms[i] = op->tune_ms[i];
    return LS_OK;
}

ls_status ls_op_setup_times(const ls_op* op, double* t4) {
    if (!op || !t4) return fail(LS_EINVAL, "null argument");
    for (int i = 0; i < 4; ++i) t4[i] = op->t_setup[i];
    return LS_OK;
}

ls_status ls_op_set_timing(ls_op* op, int32_t on) {
    if (!op) return fail(LS_EINVAL, "null op");
    CK(cudaStreamSynchronize(op->stream));
    for (auto& e : op->ev) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    op->ev.clear();
    op->ev_kind.clear();
    op->timing = on != 0;
    op->launches = 0;
    op->pairsum_launches = 0;
    return LS_OK;
}

ls_status ls_op_stats(ls_op* op, double* pairsum_ms, int64_t* pairsum_launches, int64_t* launches) {
    if (!op) return fail(LS_EINVAL, "null op");
    CK(cudaStreamSynchronize(op->stream));
    double tot = 0.0;
    for (auto& e : op->ev) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e.first, e.second));
        tot += ms;
    }
    if (pairsum_ms) *pairsum_ms = tot;
    if (pairsum_launches) *pairsum_launches = op->timing ? (int64_t)op->ev.size() : op->pairsum_launches;
    if (launches) *launches = op->launches;
    return LS_OK;
}

ls_status ls_op_stats_kind(ls_op* op, int32_t kind, double* pairsum_ms, int64_t* pairsum_launches) {
    if (!op) return fail(LS_EINVAL, "null op");
    CK(cudaStreamSynchronize(op->stream));
    double tot = 0.0;
    int64_t cnt = 0;
    for (size_t i = 0; i < op->ev.size(); ++i) {
        if (op->ev_kind[i] != kind) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, op->ev[i].first, op->ev[i].second));
        tot += ms;
        cnt++;
    }
    if (pairsum_ms) *pairsum_ms = tot;
    if (pairsum_launches) *pairsum_launches = cnt;
    return LS_OK;
}

ls_status ls_probe_fp64(double* gflops, void* stream) {
    if (!gflops) return fail(LS_EINVAL, "null argument");
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf<double> sink;
    CK(sink.alloc(1));
    const int threads = 256, blocks = nsm * 8, iters = 1 << 14;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    k_probe_dfma<<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7, sink.p);   // warm-up
    CK(cudaEventRecord(e0, st));
    k_probe_dfma<<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7, sink.p);
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *gflops = 2.0 * 8.0 * iters * (double)threads * blocks / (ms * 1e-3) / 1e9;
    return LS_OK;
}

ls_status ls_hankel0_dev(int64_t n, const double* z_dev, void* h_dev, void* stream) {
    if (n < 0 || (n > 0 && (!z_dev || !h_dev))) return fail(LS_EINVAL, "null argument");
    if (n == 0) return LS_OK;
    k_hankel0<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, z_dev, (double2*)h_dev);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return LS_OK;
}

}  // extern "C"
