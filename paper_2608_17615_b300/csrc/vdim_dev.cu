// Device build of the VDIM near/self correction dV (Eq. DIM_decomp, local-patch form).
//
// For target node x_j and one subdomain patch P with interpolation element tau:
//     dV_jq = E_jq - N_jq,
//     E_jq = -chi Phi_q(x_j) + int_{dP} [G dPhi_q/dn - Phi_q dG/dn_y] ds_y,
//     N_jq = sum_{n in P, n != j} G(x_j, y_n) w_n L_q(y_n),
// with L_q the Lagrange basis of tau's 15 nodes and Phi_q = L_q/k^2 - Lap L_q/k^4 +
// Lap^2 L_q/k^6 written in scaled monomials, E = Phi^T Mo and N = C^T Mn from the
// monomial moments
//     Mo_a = int_{dP} [G dm_a/dn - m_a dG/dn] ds,   Mn_a = sum_n G w_n m_a(y_n).
// dV is a small difference of two large numbers, so the moments are accumulated in
// double-double arithmetic (dd.cuh): the boundary points (straight segments or the
// exact polar-curve arcs), G = (i/4) H0^(1)(k r) and dG/dn from the ascending series
// of J0, J1, Y0, Y1 (Abramowitz & Stegun 9.1.10-9.1.13, valid and accurate in DD for
// k r <= 32), and the sums.  The work list (patches, boundary panels from the same
// dyadic refinement as the host build) and the per-element coefficient matrices
// (long double) come from the host; one warp takes one (target, patch) block: 32 lanes
// evaluate the 32 Gauss-Legendre points of a panel (or 32 patch nodes), then 30 lanes
// accumulate the 15 complex moments.  Blocks whose patch reaches k r > 32 are flagged
// and rebuilt by the host routine.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <string>
#include <vector>

#include "dd.cuh"
#include "ls_internal.h"

namespace {

constexpr int VD_WARPS = 4;
constexpr double VD_ZMAX = 32.0;

struct VdBlock {
    int target, tau, own, pad;
    int64_t e0, e1, p0, p1;
};

struct VdPanel {
    int edge, pad;
    DD a, b;
};

struct VdCtx {
    DD cx, cy, invh;
    DD C[225], Phi[225];          // [monomial a][node q]
};

struct VdPoint {
    DD gr, gi, dr, di;            // G w and dG/dn w (real, imaginary)
    DD m[15], dn[15];             // monomials and their normal derivatives
};

// monomial exponents in the order of the host build: by degree, then by the power of s2
__constant__ int vd_ea[15] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0};
__constant__ int vd_eb[15] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4};

__device__ __forceinline__ void powers(DD s, DD* p) {
    p[0] = dd(1.0);
    p[1] = s;
    p[2] = dd_mul(s, s);
    p[3] = dd_mul(p[2], s);
    p[4] = dd_mul(p[2], p[2]);
}

// J0, Y0 (and J1, Y1 when want1) at z > 0 by the ascending series
__device__ void bessel01_dd(DD z, bool want1, DD& j0, DD& y0, DD& j1, DD& y1) {
    const DD mq = dd_neg(dd_ldexp(dd_mul(z, z), -2));
    DD t0 = dd(1.0), t1 = dd(1.0), s0 = dd(1.0), s1 = dd(1.0), a0 = dd(0.0), a1 = dd(1.0);
#pragma unroll 1
    for (int k = 1; k <= DD_NSERIES; ++k) {
        t0 = dd_mul(dd_mul(t0, mq), dd_rk2[k]);
        s0 = dd_add(s0, t0);
        a0 = dd_add(a0, dd_mul(dd_hk[k], t0));
        if (want1) {
            t1 = dd_mul(dd_mul(t1, mq), dd_rkk1[k]);
            s1 = dd_add(s1, t1);
            a1 = dd_add(a1, dd_mul(dd_hh[k], t1));
        }
        if (fabs(t0.h) < 1e-36 && (!want1 || fabs(t1.h) < 1e-36)) break;
    }
    const DD two_pi_inv = DD_2_PI;                   // 2 / pi
    const DD euler = DD_EULER;
    const DD L = dd_add(dd_log(dd_ldexp(z, -1)), euler);
    j0 = s0;
    y0 = dd_mul(two_pi_inv, dd_sub(dd_mul(L, j0), a0));
    if (want1) {
        j1 = dd_mul(s1, dd_ldexp(z, -1));
        // Y1 = -2/(pi z) + (2/pi) L J1 - z/(2 pi) a1
        y1 = dd_sub(dd_mul(two_pi_inv, dd_mul(L, j1)), dd_div(two_pi_inv, z));
        y1 = dd_sub(y1, dd_mul(dd_ldexp(two_pi_inv, -2), dd_mul(z, a1)));
    }
}

// point and derivative (times the parameter length) of edge 3 el + le at parameter t
__device__ void edge_point_dd(int edge, DD t, const double2* vxy, const int* tri, const int* ecurve,
                              const double2* etheta, const double* curves, DD& x, DD& y, DD& dx, DD& dy) {
    const int el = edge / 3, le = edge - 3 * el;
    const int c = ecurve[edge];
    if (c < 0) {
        const double2 A = vxy[tri[3 * el + le]], B = vxy[tri[3 * el + (le + 1) % 3]];
        dx = two_sum(B.x, -A.x);
        dy = two_sum(B.y, -A.y);
        x = dd_add(dd(A.x), dd_mul(t, dx));
        y = dd_add(dd(A.y), dd_mul(t, dy));
        return;
    }
    const double* C = curves + 6 * c;            // (cx, cy, R, a, m, phi)
    const double2 th01 = etheta[edge];
    const DD dth = two_sum(th01.y, -th01.x);
    const DD th = dd_add(dd(th01.x), dd_mul(t, dth));
    const DD ang = dd_add_d(dd_mul_d(th, C[4]), C[5]);
    DD sa, ca, st, ct;
    dd_sincos(ang, sa, ca);
    dd_sincos(th, st, ct);
    const DD rr = dd_mul_d(dd_add_d(dd_mul_d(ca, C[3]), 1.0), C[2]);
    const DD dr = dd_neg(dd_mul_d(dd_mul_d(dd_mul_d(sa, C[2]), C[3]), C[4]));
    x = dd_add_d(dd_mul(rr, ct), C[0]);
    y = dd_add_d(dd_mul(rr, st), C[1]);
    dx = dd_mul(dd_sub(dd_mul(dr, ct), dd_mul(rr, st)), dth);
    dy = dd_mul(dd_add(dd_mul(dr, st), dd_mul(rr, ct)), dth);
}

__global__ void __launch_bounds__(32 * VD_WARPS) k_vdim(int64_t b_begin, int64_t b_end, const VdBlock* __restrict__ blocks,
                                                       const VdPanel* __restrict__ pans, const int* __restrict__ elems,
                                                       const double2* __restrict__ nodes, const double* __restrict__ wts,
                                                       const double2* __restrict__ vxy, const int* __restrict__ tri,
                                                       const int* __restrict__ ecurve, const double2* __restrict__ etheta,
                                                       const double* __restrict__ curves, const VdCtx* __restrict__ ctx,
                                                       DD kk, const DD* __restrict__ glx, const DD* __restrict__ glw,
                                                       double2* __restrict__ vals, int* __restrict__ flag) {
    extern __shared__ VdPoint vsh[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = b_begin + (int64_t)blockIdx.x * VD_WARPS + warp;
    if (b >= b_end) return;
    VdPoint* pts = vsh + warp * 32;
    const VdBlock B = blocks[b];
    const VdCtx& X = ctx[B.tau];
    const double2 xj2 = nodes[B.target];
    const DD xj = dd(xj2.x), yj = dd(xj2.y);
    const DD k4 = dd_ldexp(kk, -2);
    const int a = lane % 15, part = lane / 15;          // moment handled in phase B (lanes < 30)
    DD accE = dd(0.0), accN = dd(0.0);
    bool far = false;
    // boundary moments, panel by panel
    for (int64_t p = B.p0; p < B.p1; ++p) {
        const VdPanel P = pans[p];
        const DD len = dd_sub(P.b, P.a);
        const DD t = dd_add(P.a, dd_mul(len, glx[lane]));
        const DD wt = dd_mul(len, glw[lane]);
        DD x, y, dx, dy;
        edge_point_dd(P.edge, t, vxy, tri, ecurve, etheta, curves, x, y, dx, dy);
        const DD nx = dy, ny = dd_neg(dx);                  // outward normal times |y'|
        const DD rx = dd_sub(x, xj), ry = dd_sub(y, yj);
        const DD r = dd_sqrt(dd_add(dd_mul(rx, rx), dd_mul(ry, ry)));
        const DD z = dd_mul(kk, r);
        VdPoint& Q = pts[lane];
        if (z.h > VD_ZMAX) {
            far = true;
            Q.gr = Q.gi = Q.dr = Q.di = dd(0.0);
        } else {
            DD j0, y0, j1, y1;
            bessel01_dd(z, true, j0, y0, j1, y1);
            // G = (i/4)(J0 + i Y0);  dG/dn = -(i k / 4)(J1 + i Y1) (r . n) / r
            const DD proj = dd_div(dd_add(dd_mul(rx, nx), dd_mul(ry, ny)), r);
            Q.gr = dd_neg(dd_ldexp(dd_mul(y0, wt), -2));
            Q.gi = dd_ldexp(dd_mul(j0, wt), -2);
            const DD kp = dd_mul(dd_mul(k4, proj), wt);
            Q.dr = dd_mul(kp, y1);
            Q.di = dd_neg(dd_mul(kp, j1));
        }
        DD p1[5], p2[5];
        powers(dd_mul(dd_sub(x, X.cx), X.invh), p1);
        powers(dd_mul(dd_sub(y, X.cy), X.invh), p2);
#pragma unroll
        for (int i = 0; i < 15; ++i) {
            const int ea = vd_ea[i], eb = vd_eb[i];
            Q.m[i] = dd_mul(p1[ea], p2[eb]);
            DD g = dd(0.0);
            if (ea) g = dd_mul(dd_mul_d(dd_mul(p1[ea - 1], p2[eb]), (double)ea), nx);
            if (eb) g = dd_add(g, dd_mul(dd_mul_d(dd_mul(p1[ea], p2[eb - 1]), (double)eb), ny));
            Q.dn[i] = dd_mul(g, X.invh);
        }
        __syncwarp();
        if (lane < 30) {
            for (int i = 0; i < 32; ++i) {
                const VdPoint& R = pts[i];
                const DD g = part ? R.gi : R.gr, d = part ? R.di : R.dr;
                accE = dd_add(accE, dd_sub(dd_mul(g, R.dn[a]), dd_mul(d, R.m[a])));
            }
        }
        __syncwarp();
    }
    // plain-quadrature moments over the patch nodes (the target itself excluded)
    const int64_t total = (B.e1 - B.e0) * lsgpu::NQ_ELEM;
    for (int64_t base = 0; base < total; base += 32) {
        const int64_t idx = base + lane;
        VdPoint& Q = pts[lane];
        Q.gr = Q.gi = dd(0.0);
        int n = -1;
        if (idx < total) n = elems[B.e0 + idx / lsgpu::NQ_ELEM] * lsgpu::NQ_ELEM + (int)(idx % lsgpu::NQ_ELEM);
        if (n >= 0 && n != B.target) {
            const double2 yn = nodes[n];
            const DD rx = two_sum(yn.x, -xj2.x), ry = two_sum(yn.y, -xj2.y);
            const DD r = dd_sqrt(dd_add(dd_mul(rx, rx), dd_mul(ry, ry)));
            const DD z = dd_mul(kk, r);
            if (z.h > VD_ZMAX) {
                far = true;
            } else {
                DD j0, y0, j1, y1;
                bessel01_dd(z, false, j0, y0, j1, y1);
                Q.gr = dd_neg(dd_ldexp(dd_mul_d(y0, wts[n]), -2));
                Q.gi = dd_ldexp(dd_mul_d(j0, wts[n]), -2);
            }
            DD p1[5], p2[5];
            powers(dd_mul(dd_sub(dd(yn.x), X.cx), X.invh), p1);
            powers(dd_mul(dd_sub(dd(yn.y), X.cy), X.invh), p2);
#pragma unroll
            for (int i = 0; i < 15; ++i) Q.m[i] = dd_mul(p1[vd_ea[i]], p2[vd_eb[i]]);
        } else {
#pragma unroll
            for (int i = 0; i < 15; ++i) Q.m[i] = dd(0.0);
        }
        __syncwarp();
        if (lane < 30) {
            const int cnt = (int)(total - base < 32 ? total - base : 32);
            for (int i = 0; i < cnt; ++i) {
                const VdPoint& R = pts[i];
                accN = dd_add(accN, dd_mul(part ? R.gi : R.gr, R.m[a]));
            }
        }
        __syncwarp();
    }
    far = __any_sync(0xffffffffu, far);
    // E = Phi^T Mo - chi Phi(x_j),  N = C^T Mn,  dV = E - N
    DD* mo = &pts[0].gr;                 // reuse the point buffer: mo[2 a + part], mn at +30
    if (lane < 30) {
        mo[2 * a + part] = accE;
        mo[30 + 2 * a + part] = accN;
    }
    __syncwarp();
    if (lane < 30) {
        const int q = a;
        DD E = dd(0.0), N = dd(0.0);
        for (int i = 0; i < 15; ++i) {
            E = dd_add(E, dd_mul(X.Phi[i * 15 + q], mo[2 * i + part]));
            N = dd_add(N, dd_mul(X.C[i * 15 + q], mo[30 + 2 * i + part]));
        }
        if (B.own && part == 0) {
            DD p1[5], p2[5];
            powers(dd_mul(dd_sub(xj, X.cx), X.invh), p1);
            powers(dd_mul(dd_sub(yj, X.cy), X.invh), p2);
            DD phi = dd(0.0);
            for (int i = 0; i < 15; ++i) phi = dd_add(phi, dd_mul(dd_mul(p1[vd_ea[i]], p2[vd_eb[i]]), X.Phi[i * 15 + q]));
            E = dd_sub(E, phi);
        }
        const double v = dd_sub(E, N).h;
        double* out = reinterpret_cast<double*>(vals + b * 15 + q);
        out[part] = v;
    }
    if (lane == 0) flag[b] = far ? 1 : 0;
}

inline DD to_dd(long double x) {
    const double h = (double)x;
    return DD{h, (double)(x - (long double)h)};
}

template <typename T>
struct DBuf {
    T* p = nullptr;
    ~DBuf() { if (p) cudaFree(p); }
    cudaError_t up(const std::vector<T>& v) {
        if (v.empty()) return cudaSuccess;
        cudaError_t e = cudaMalloc(&p, sizeof(T) * v.size());
        if (e != cudaSuccess) return e;
        return cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    }
};

#define VCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return std::string(#call) + ": " + cudaGetErrorString(e_);  \
    } while (0)

}  // namespace

namespace lsgpu {

std::string build_correction_device(const HostMesh& M, double k, double kappa, void* stream, CsrC& out,
                                    int64_t* host_blocks) {
    cudaStream_t st = (cudaStream_t)stream;
    CorrPlan P;
    std::string err = plan_correction(M, kappa, P);
    if (!err.empty()) return err;
    const int64_t nb = (int64_t)P.target.size();
    // per-element coefficient matrices (host, long double)
    std::vector<VdCtx> ctx(M.nt);
    int bad = -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int t = 0; t < M.nt; ++t) {
        long double c3[3], C[225], Phi[225];
        if (!poly_context(M, t, k, c3, C, Phi)) {
#pragma omp critical
            bad = t;
            continue;
        }
        VdCtx& X = ctx[t];
        X.cx = to_dd(c3[0]);
        X.cy = to_dd(c3[1]);
        X.invh = to_dd(c3[2]);
        for (int i = 0; i < 225; ++i) {
            X.C[i] = to_dd(C[i]);
            X.Phi[i] = to_dd(Phi[i]);
        }
    }
    if (bad >= 0) return "singular interpolation matrix of element " + std::to_string(bad);
    std::vector<VdBlock> blk(nb);
    for (int64_t b = 0; b < nb; ++b)
        blk[b] = VdBlock{P.target[b], P.tau[b], P.own[b], 0, P.elem_off[b], P.elem_off[b + 1], P.pan_off[b], P.pan_off[b + 1]};
    std::vector<VdPanel> pan(P.pan_edge.size());
    for (size_t i = 0; i < pan.size(); ++i) pan[i] = VdPanel{P.pan_edge[i], 0, to_dd(P.pan_a[i]), to_dd(P.pan_b[i])};
    long double gx[32], gw[32];
    gl32_unit(gx, gw);
    std::vector<DD> glx(32), glw(32);
    for (int i = 0; i < 32; ++i) { glx[i] = to_dd(gx[i]); glw[i] = to_dd(gw[i]); }
    std::vector<double2> nodes(M.nq), vxy(M.nv), eth(3 * (size_t)M.nt);
    for (int i = 0; i < M.nq; ++i) nodes[i] = make_double2(M.nodes[2 * i], M.nodes[2 * i + 1]);
    for (int i = 0; i < M.nv; ++i) vxy[i] = make_double2(M.vxy[2 * i], M.vxy[2 * i + 1]);
    for (size_t i = 0; i < eth.size(); ++i) eth[i] = make_double2(M.etheta[2 * i], M.etheta[2 * i + 1]);
    DBuf<VdBlock> dblk;
    DBuf<VdPanel> dpan;
    DBuf<int> delems, dtri, dcurve, dflag;
    DBuf<double2> dnodes, dvxy, deth, dvals;
    DBuf<double> dw, dcurves;
    DBuf<VdCtx> dctx;
    DBuf<DD> dglx, dglw;
    VCK(dblk.up(blk));
    VCK(dpan.up(pan));
    VCK(delems.up(std::vector<int>(P.elems.begin(), P.elems.end())));
    VCK(dtri.up(M.tri));
    VCK(dcurve.up(M.ecurve));
    VCK(dnodes.up(nodes));
    VCK(dvxy.up(vxy));
    VCK(deth.up(eth));
    VCK(dw.up(M.w));
    VCK(dcurves.up(M.curves.empty() ? std::vector<double>(6, 0.0) : M.curves));
    VCK(dctx.up(ctx));
    VCK(dglx.up(glx));
    VCK(dglw.up(glw));
    VCK(cudaMalloc(&dvals.p, sizeof(double2) * 15 * std::max<int64_t>(nb, 1)));
    VCK(cudaMalloc(&dflag.p, sizeof(int) * std::max<int64_t>(nb, 1)));
    const size_t smem = sizeof(VdPoint) * 32 * VD_WARPS;
    VCK(cudaFuncSetAttribute(k_vdim, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const DD kk = DD{k, 0.0};
    const int64_t chunk = 1 << 16;
    for (int64_t b0 = 0; b0 < nb; b0 += chunk) {
        const int64_t b1 = std::min(nb, b0 + chunk);
        const unsigned grid = (unsigned)((b1 - b0 + VD_WARPS - 1) / VD_WARPS);
        k_vdim<<<grid, 32 * VD_WARPS, smem, st>>>(b0, b1, dblk.p, dpan.p, delems.p, dnodes.p, dw.p, dvxy.p, dtri.p,
                                                  dcurve.p, deth.p, dcurves.p, dctx.p, kk, dglx.p, dglw.p, dvals.p,
                                                  dflag.p);
        VCK(cudaGetLastError());
    }
    std::vector<std::complex<double>> vals(15 * (size_t)nb);
    std::vector<int> flag(nb);
    VCK(cudaMemcpyAsync(vals.data(), dvals.p, sizeof(double2) * 15 * nb, cudaMemcpyDeviceToHost, st));
    VCK(cudaMemcpyAsync(flag.data(), dflag.p, sizeof(int) * nb, cudaMemcpyDeviceToHost, st));
    VCK(cudaStreamSynchronize(st));
    // blocks whose patch reaches beyond the series range: the host routine
    std::vector<int64_t> redo;
    for (int64_t b = 0; b < nb; ++b)
        if (flag[b]) redo.push_back(b);
    int failed = -1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < (int64_t)redo.size(); ++i) {
        const int64_t b = redo[i];
        std::vector<int> patch(P.elems.begin() + P.elem_off[b], P.elems.begin() + P.elem_off[b + 1]);
        if (!correction_block_host(M, P.target[b], k, patch, P.tau[b], P.own[b] != 0, vals.data() + 15 * b)) {
#pragma omp critical
            failed = (int)b;
        }
    }
    if (failed >= 0) return "singular interpolation matrix in block " + std::to_string(failed);
    if (host_blocks) *host_blocks = (int64_t)redo.size();
    const int nq = M.nq;
    out.rowptr.assign(nq + 1, 0);
    for (int j = 0; j < nq; ++j) out.rowptr[j + 1] = 15 * P.row_blocks[j + 1];
    out.cols.resize(15 * (size_t)nb);
    out.vals = std::move(vals);
    for (int64_t b = 0; b < nb; ++b)
        for (int q = 0; q < 15; ++q) out.cols[15 * b + q] = P.tau[b] * NQ_ELEM + q;
    return "";
}

}  // namespace lsgpu
