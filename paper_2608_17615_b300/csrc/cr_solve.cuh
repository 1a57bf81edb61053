// Block cyclic reduction for the block-tridiagonal Cartesian matrix C = A L^(C)
// (Eq. LC_def) of the sparsifying preconditioner, S = C^{-1} A (Eq. S_minus_I).
//
// C has ny block rows of nx x nx blocks (grid row b couples only to rows b-1, b, b+1):
//     L_b x_{b-1} + D_b x_b + U_b x_{b+1} = t_b,
// with tridiagonal L_b, D_b, U_b read from the band storage cband[ny][9][nx].
// The paper factors C with nested dissection (a CPU sparse direct solver); on the
// GPU a direct solve must stream dense factor blocks at HBM speed, and a block LU
// sweep does that one block row at a time (ny dependent steps).  Cyclic reduction
// removes the odd-numbered block rows at every level,
//     z_i = D_i^{-1} t_i                                 (odd i)
//     t'_j = t_j - L_j z_{j-1} - U_j z_{j+1}             (even j)
//     L'_j = -L_j gamma_{j-1},  U'_j = -U_j delta_{j+1},
//     D'_j = D_j - L_j delta_{j-1} - U_j gamma_{j+1},    gamma_i = D_i^{-1} L_i, delta_i = D_i^{-1} U_i,
// leaving a block-tridiagonal system on the even rows; after ceil(log2 ny) levels
// one block remains, and the odd rows come back from
//     x_i = z_i - gamma_i x_{i-1} - delta_i x_{i+1}.
// Every level is a batch of independent dense matrix-vector products, so the whole
// solve is 3 log2(ny) + 1 wide launches instead of 2 ny - 1 narrow ones.  The
// transposed solve C^T x = t (for P^T) uses the same blocks transposed:
//     t'_j = t_j - gamma_{j+1}^T t_{j+1} - delta_{j-1}^T t_{j-1}            (even j)
//     x_i = D_i^{-T} (t_i - L_{i+1}^T x_{i+1} - U_{i-1}^T x_{i-1})          (odd i)
// (the odd-even elimination is a block LU of the permuted matrix; transposing it
// swaps the roles of gamma/delta and L/U).
//
// Storage: level 0 keeps L, U in the band; every level stores D_i^{-1}, gamma_i,
// delta_i for its odd rows and (from level 1 on, where they are dense) L_j, U_j for
// its even rows, each also transposed: about 8 ny dense blocks of nx^2 complex128.
#pragma once

struct CRJob {                 // y = base - (M1 v1 + M2 v2), or y = M1 v1 when base is null
    double2* y;
    const double2* base;
    const double2* M1;
    const double2* v1;
    const double2* M2;
    const double2* v2;
};

struct CRTriJob {              // level 0: y = base - (L_bL or L_bL^T) vL - (U_bU or U_bU^T) vU from the band
    double2* y;
    const double2* base;
    const double2* vL;
    const double2* vU;
    int bL, bU;                // block rows of C whose L / U band is used (-1: none)
};

#define CR_WARPS 8
#define CR_ROWS_PER_WARP 2

// Dense block matrix-vector products, row-major nx x nx blocks; one job per
// grid.y, CR_WARPS * CR_ROWS_PER_WARP rows per CTA along grid.x, RG right-hand
// sides per CTA along grid.z (vector r of a job sits at offset r * svec).
template <int RG>
__global__ void __launch_bounds__(32 * CR_WARPS) k_cr_mv(int nx, int R, size_t svec, const CRJob* __restrict__ jobs) {
    extern __shared__ double2 crsh[];                    // [RG][2][nx]
    const CRJob J = jobs[blockIdx.y];
    const int r0 = blockIdx.z * RG;
    const int nr = min(RG, R - r0);
    for (int i = threadIdx.x; i < RG * nx; i += blockDim.x) {
        const int r = i / nx, c = i - r * nx;
        const bool ok = r < nr;
        crsh[(2 * r) * nx + c] = ok ? J.v1[(size_t)(r0 + r) * svec + c] : make_double2(0.0, 0.0);
        crsh[(2 * r + 1) * nx + c] = (ok && J.M2) ? J.v2[(size_t)(r0 + r) * svec + c] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = 0; q < CR_ROWS_PER_WARP; ++q) {
        const int row = (blockIdx.x * CR_WARPS + warp) * CR_ROWS_PER_WARP + q;
        if (row >= nx) break;
        double ar[RG], ai[RG];
#pragma unroll
        for (int r = 0; r < RG; ++r) { ar[r] = 0.0; ai[r] = 0.0; }
        const double2* m1 = J.M1 + (size_t)row * nx;
#pragma unroll 4
        for (int c = lane; c < nx; c += 32) {
            const double2 a = m1[c];
#pragma unroll
            for (int r = 0; r < RG; ++r) {
                const double2 v = crsh[(2 * r) * nx + c];
                ar[r] = fma(a.x, v.x, fma(-a.y, v.y, ar[r]));
                ai[r] = fma(a.x, v.y, fma(a.y, v.x, ai[r]));
            }
        }
        if (J.M2) {
            const double2* m2 = J.M2 + (size_t)row * nx;
#pragma unroll 4
            for (int c = lane; c < nx; c += 32) {
                const double2 a = m2[c];
#pragma unroll
                for (int r = 0; r < RG; ++r) {
                    const double2 v = crsh[(2 * r + 1) * nx + c];
                    ar[r] = fma(a.x, v.x, fma(-a.y, v.y, ar[r]));
                    ai[r] = fma(a.x, v.y, fma(a.y, v.x, ai[r]));
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RG; ++r) {
            for (int o = 16; o > 0; o >>= 1) {
                ar[r] += __shfl_down_sync(0xffffffffu, ar[r], o);
                ai[r] += __shfl_down_sync(0xffffffffu, ai[r], o);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int r = 0; r < RG; ++r) {
                if (r >= nr) break;
                const size_t o = (size_t)(r0 + r) * svec + row;
                if (J.base) {
                    const double2 b = J.base[o];
                    J.y[o] = make_double2(b.x - ar[r], b.y - ai[r]);
                } else {
                    J.y[o] = make_double2(ar[r], ai[r]);
                }
            }
        }
    }
}

// The same products with the factor blocks stored as double-float pairs (hi.re, hi.im,
// lo.re, lo.im per complex entry: the 16 bytes of a complex128) and double-float arithmetic
// on the FP32 pipe, single right-hand side: B300's FP64 pipe caps the complex128 product at
// about a third of HBM speed, the double-float one reads the same bytes with FP32
// instructions (rounding ~1e-13 instead of ~1e-16, far below what the forms that take it,
// the FP32 and mixed solves, can see).  Vectors stay FP64.
struct CRJobDF {
    double2* y;
    const double2* base;
    const float4* M1;
    const double2* v1;
    const float4* M2;
    const double2* v2;
};

__device__ __forceinline__ void cr_df_fast(float& h, float& l) {      // renormalise |h| >= |l|
    const float s = h + l;
    l = l - (s - h);
    h = s;
}
__device__ __forceinline__ void cr_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bv = s - a;
    const float av = s - bv;
    e = (a - av) + (b - bv);
}
// (rh, rl) + i (ih, il) += a * v, a and v double-float complex as (hi.re, hi.im, lo.re, lo.im);
// products to first order (high product, FMA residual, cross terms), high parts by TwoSum,
// every residual into the low word
__device__ __forceinline__ void cr_df_cmac(float4 a, float4 v, float& rh, float& rl, float& ih, float& il) {
    const float p1 = a.x * v.x, p2 = a.y * v.y, p3 = a.x * v.y, p4 = a.y * v.x;
    float e1 = fmaf(a.x, v.x, -p1), e2 = fmaf(a.y, v.y, -p2), e3 = fmaf(a.x, v.y, -p3), e4 = fmaf(a.y, v.x, -p4);
    e1 = fmaf(a.z, v.x, fmaf(a.x, v.z, e1));
    e2 = fmaf(a.w, v.y, fmaf(a.y, v.w, e2));
    e3 = fmaf(a.z, v.y, fmaf(a.x, v.w, e3));
    e4 = fmaf(a.w, v.x, fmaf(a.y, v.z, e4));
    float t, err;
    cr_two_sum(rh, p1, t, err);
    rl += err + e1;
    cr_two_sum(t, -p2, rh, err);
    rl += err - e2;
    cr_two_sum(ih, p3, t, err);
    il += err + e3;
    cr_two_sum(t, p4, ih, err);
    il += err + e4;
}

__global__ void __launch_bounds__(32 * CR_WARPS) k_cr_mv_df(int nx, const CRJobDF* __restrict__ jobs) {
    extern __shared__ float4 crshdf[];                   // [2][nx] double-float vectors
    const CRJobDF J = jobs[blockIdx.y];
    for (int c = threadIdx.x; c < nx; c += blockDim.x) {
        const double2 a = J.v1[c];
        const float ah = (float)a.x, bh = (float)a.y;
        crshdf[c] = make_float4(ah, bh, (float)(a.x - (double)ah), (float)(a.y - (double)bh));
        const double2 b = J.M2 ? J.v2[c] : make_double2(0.0, 0.0);
        const float ch = (float)b.x, dh = (float)b.y;
        crshdf[nx + c] = make_float4(ch, dh, (float)(b.x - (double)ch), (float)(b.y - (double)dh));
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the warp's CR_ROWS_PER_WARP (= 2) rows side by side: two independent accumulation
    // chains and twice the loads in flight per column step
    static_assert(CR_ROWS_PER_WARP == 2, "k_cr_mv_df interleaves two rows per warp");
    const int row0 = (blockIdx.x * CR_WARPS + warp) * CR_ROWS_PER_WARP;
    if (row0 >= nx) return;
    const bool two = row0 + 1 < nx;
    const int row1 = two ? row0 + 1 : row0;
    float r0h = 0.f, r0l = 0.f, i0h = 0.f, i0l = 0.f, r1h = 0.f, r1l = 0.f, i1h = 0.f, i1l = 0.f;
    for (int m = 0; m < 2; ++m) {
        const float4* M = m ? J.M2 : J.M1;
        if (!M) break;
        const float4* a0 = M + (size_t)row0 * nx;
        const float4* a1 = M + (size_t)row1 * nx;
        const float4* v = crshdf + m * nx;
        // nx / 32 terms per lane and matrix (8 at 256 nodes, 16 at 512): the low words stay
        // within a few ulps of the high ones until the normalisation after the matrix
#pragma unroll 8
        for (int c = lane; c < nx; c += 32) {
            const float4 x0 = a0[c], x1 = a1[c], vv = v[c];
            cr_df_cmac(x0, vv, r0h, r0l, i0h, i0l);
            cr_df_cmac(x1, vv, r1h, r1l, i1h, i1l);
        }
        cr_df_fast(r0h, r0l); cr_df_fast(i0h, i0l);
        cr_df_fast(r1h, r1l); cr_df_fast(i1h, i1l);
    }
    // warp sums in FP64 of the lanes' double-float partials
    double s0r = (double)r0h + (double)r0l, s0i = (double)i0h + (double)i0l;
    double s1r = (double)r1h + (double)r1l, s1i = (double)i1h + (double)i1l;
    for (int o = 16; o > 0; o >>= 1) {
        s0r += __shfl_down_sync(0xffffffffu, s0r, o);
        s0i += __shfl_down_sync(0xffffffffu, s0i, o);
        s1r += __shfl_down_sync(0xffffffffu, s1r, o);
        s1i += __shfl_down_sync(0xffffffffu, s1i, o);
    }
    if (lane == 0) {
        const int rows[2] = {row0, row1};
        const double sr[2] = {s0r, s1r}, si[2] = {s0i, s1i};
        for (int q = 0; q < (two ? 2 : 1); ++q) {
            if (J.base) {
                const double2 b = J.base[rows[q]];
                J.y[rows[q]] = make_double2(b.x - sr[q], b.y - si[q]);
            } else {
                J.y[rows[q]] = make_double2(sr[q], si[q]);
            }
        }
    }
}

// Level-0 updates with the tridiagonal band blocks of C (entry (a, a + da) of
// L_b at cband[(9 b + da + 1) nx + a], of U_b at cband[(9 b + 6 + da + 1) nx + a]).
// transposed = 0: y_a = base_a - sum_da L(a, a+da) vL_{a+da} - sum_da U(a, a+da) vU_{a+da}
// transposed = 1: y_c = base_c - sum_da L(c-da, c) vL_{c-da} - sum_da U(c-da, c) vU_{c-da}
__global__ void k_cr_tri(int nx, int R, size_t svec, const double2* __restrict__ cband, const CRTriJob* __restrict__ jobs,
                         int transposed) {
    const CRTriJob J = jobs[blockIdx.y];
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nx) return;
    for (int r = 0; r < R; ++r) {
        const size_t o = (size_t)r * svec;
        double2 acc = J.base[o + a];
        for (int side = 0; side < 2; ++side) {
            const int bb = side ? J.bU : J.bL;
            if (bb < 0) continue;
            const double2* v = (side ? J.vU : J.vL) + o;
            const double2* band = cband + ((size_t)bb * 9 + (side ? 6 : 0)) * nx;
#pragma unroll
            for (int da = -1; da <= 1; ++da) {
                const int c = transposed ? a - da : a + da;
                if (c < 0 || c >= nx) continue;
                const double2 e = band[(size_t)(da + 1) * nx + (transposed ? c : a)];
                const double2 x = v[c];
                acc.x -= e.x * x.x - e.y * x.y;
                acc.y -= e.x * x.y + e.y * x.x;
            }
        }
        J.y[o + a] = acc;
    }
}

// Dense row-major block (r, c) <- band block of C (which = 0: L_b, 1: D_b, 2: U_b).
__global__ void k_cr_expand(int nx, const double2* __restrict__ cband, const int* __restrict__ blk, int which,
                            double2* const* __restrict__ out) {
    const int r = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nx) return;
    const int b = blk[blockIdx.z];
    const int da = c - r;
    double2 v = make_double2(0.0, 0.0);
    if (da >= -1 && da <= 1) v = cband[((size_t)b * 9 + 3 * which + da + 1) * nx + r];
    out[blockIdx.z][(size_t)r * nx + c] = v;
}

// out_i = in_i^T for a list of row-major nx x nx blocks
__global__ void k_cr_transpose(int nx, const double2* const* __restrict__ in, double2* const* __restrict__ out) {
    __shared__ double2 t[32][33];
    const double2* src = in[blockIdx.z];
    double2* dst = out[blockIdx.z];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = y0 + i, c = x0 + threadIdx.x;
        if (r < nx && c < nx) t[i][threadIdx.x] = src[(size_t)r * nx + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = x0 + i, c = y0 + threadIdx.x;
        if (r < nx && c < nx) dst[(size_t)r * nx + c] = t[threadIdx.x][i];
    }
}

__global__ void k_cr_identity(int nx, double2* const* __restrict__ out) {
    const int r = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nx) out[blockIdx.z][(size_t)r * nx + c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
}
