// Host setup of the Lippmann-Schwinger operator, in extended precision.
//
//  * hankel01_ld: H0^(1), H1^(1) for real z > 0 in long double (x86 80-bit):
//      z <= 6      ascending series (Abramowitz & Stegun 9.1.10-9.1.13)
//      6 < z < 30  Miller backward recurrence normalised by J0 + 2 sum J_2k = 1,
//                  Neumann series for Y0 (A&S 9.1.88) and its derivative for Y1
//      z >= 30     Hankel asymptotic expansion (A&S 9.2.5-9.2.10)
//  * build_correction: the VDIM near/self correction dV (Eq. DIM_decomp) in the
//    local-patch form.  For target node x_j in element tau and every subdomain l
//    with elements inside the patch radius:
//      dV_jq = E_jq - N_jq,
//      E_jq = -chi Phi_q(x_j) + int_{boundary of patch} (G dPhi_q/dn - Phi_q dG/dn) ds
//      N_jq = sum_{n in patch, n != j} G(x_j, y_n) w_n L_q(y_n)
//    L_q: Lagrange basis of the interpolation element's 15 nodes (tau for the
//    own subdomain, chi = 1; the nearest element otherwise, chi = 0);
//    Phi_q = L_q/k^2 - Lap L_q/k^4 + Lap^2 L_q/k^6 solves (Lap + k^2) Phi_q = L_q.
//    Patch of target j in subdomain l: elements t of l with
//    |c_t - x_j|^2 < kappa^2 h_j^2 (c_t = ((v0 + v1) + v2) / 3, h_j^2 the largest
//    squared vertex distance of tau), plus tau itself in its own subdomain.
//    dV is a small difference of two large numbers, hence long double throughout;
//    boundary integrals use dyadic panel refinement until each panel is shorter
//    than 3/4 of its distance to the target, then 32-point Gauss-Legendre.
//  * build_grid: bilinear T_C^Q (Eq. psi_def), Approach II T_Q^C (Eq. T_H^C_def,
//    Eq. D_def), the sparsifying stencils (Eq. sparsifying_min) on the
//    neighbourhoods of Eq. cart_neighbors_LS, which the grid truncates at its
//    edges: one stencil per row class (interior, four edges, four corners) from
//    the Gram matrix of V^(C)(N(j), N(j)^c) at a representative node of the
//    class, diagonalised by Jacobi rotations, and C = A L^(C) on the 3 x 3
//    pattern (Eq. LC_def) in block-tridiagonal storage.
//    V^(C) diagonal: integral of G over the disc of area h_C^2 (the
//    Duan-Rokhlin weights of the paper are replaced by this value).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ls_internal.h"
#ifdef _OPENMP
#include <omp.h>
#endif

namespace lsgpu {

using ld = long double;
using cld = std::complex<long double>;

static const ld PI_L = 3.141592653589793238462643383279502884L;
static const ld EG_L = 0.577215664901532860606512090082402431L;

// ---------------------------------------------------------------- Hankel
struct SeriesTables {            // 1/k^2, 1/(k(k+1)), H_k and H_k + H_{k+1} for k = 1..40
    ld rk2[41], rkk1[41], hk[41], hh[41];
    SeriesTables() {
        ld h = 0;
        for (int k = 1; k <= 40; ++k) {
            rk2[k] = 1.0L / ((ld)k * k);
            rkk1[k] = 1.0L / ((ld)k * (k + 1));
            h += 1.0L / k;
            hk[k] = h;
            hh[k] = 2 * h + 1.0L / (k + 1);
        }
    }
};
static const SeriesTables& series_tables() { static SeriesTables t; return t; }

static void series01(ld z, ld& j0, ld& j1, ld& y0, ld& y1) {
    const SeriesTables& T = series_tables();
    ld q = z * z / 4;
    ld t0 = 1, t1 = 1;          // (-q)^k/(k!)^2 and (-q)^k/(k!(k+1)!)
    ld s0 = 1, s1 = 1;          // J0, J1/(z/2)
    ld hk = 0;                  // H_k
    ld a0 = 0;                  // sum_{k>=1} H_k (-q)^k/(k!)^2
    ld a1 = 1;                  // sum_{k>=0} (H_k + H_{k+1}) (-q)^k/(k!(k+1)!)
    (void)hk;
    for (int k = 1; k <= 40; ++k) {
        t0 *= -q * T.rk2[k];
        t1 *= -q * T.rkk1[k];
        s0 += t0;
        s1 += t1;
        a0 += T.hk[k] * t0;
        a1 += T.hh[k] * t1;
        if (std::fabs(t0) < 1e-24L && std::fabs(t1) < 1e-24L) break;
    }
    ld L = std::log(z / 2) + EG_L;
    j0 = s0;
    j1 = s1 * z / 2;
    y0 = (2 / PI_L) * (L * j0 - a0);
    y1 = -2 / (PI_L * z) + (2 / PI_L) * L * j1 - z / (2 * PI_L) * a1;
}

static void miller01(ld z, ld& j0, ld& j1, ld& y0, ld& y1) {
    int nstart = 2 * ((int)(z + 56) / 2);          // z < 30 here, so nstart <= 86
    ld J[96];
    for (int i = 0; i < nstart + 2; ++i) J[i] = 0.0L;
    J[nstart] = 1e-300L;
    for (int n = nstart; n >= 1; --n) {
        J[n - 1] = (2.0L * n / z) * J[n] - J[n + 1];
        if (std::fabs(J[n - 1]) > 1e300L)
            for (int i = n - 1; i <= nstart; ++i) J[i] *= 1e-300L;
    }
    ld norm = J[0];
    for (int k = 2; k <= nstart; k += 2) norm += 2 * J[k];
    for (int i = 0; i < nstart + 2; ++i) J[i] /= norm;
    ld s0 = 0, s1 = 0;
    for (int k = 1; 2 * k + 1 <= nstart + 1; ++k) {
        ld sg = (k % 2) ? -1.0L : 1.0L;
        s0 += sg * J[2 * k] / k;
        s1 += sg * (J[2 * k - 1] - J[2 * k + 1]) / k;
    }
    ld L = std::log(z / 2) + EG_L;
    j0 = J[0];
    j1 = J[1];
    y0 = (2 / PI_L) * (L * j0 - 2 * s0);
    y1 = (2 / PI_L) * (-j0 / z + L * j1 + s1);
}

static void asym01(ld z, ld& j0, ld& j1, ld& y0, ld& y1) {
    ld c = std::cos(z), s = std::sin(z);
    ld r2 = std::sqrt(0.5L);
    ld amp = std::sqrt(2 / (PI_L * z));
    ld out[4];
    for (int nu = 0; nu < 2; ++nu) {
        ld mu = 4.0L * nu * nu;
        ld P = 1, Q = 0, term = 1;
        for (int k = 1; k < 100; ++k) {
            term *= (mu - (ld)(2 * k - 1) * (2 * k - 1)) / (k * 8 * z);
            if (k % 2) Q += (((k - 1) / 2) % 2 ? -term : term);
            else       P += ((k / 2) % 2 ? -term : term);
            if (std::fabs(term) < 1e-22L) break;
        }
        ld cc, ss;   // cos, sin of z - (nu/2 + 1/4) pi
        if (nu == 0) { cc = r2 * (c + s); ss = r2 * (s - c); }
        else         { cc = r2 * (s - c); ss = -r2 * (s + c); }
        out[2 * nu] = amp * (P * cc - Q * ss);      // J_nu
        out[2 * nu + 1] = amp * (P * ss + Q * cc);  // Y_nu
    }
    j0 = out[0]; y0 = out[1]; j1 = out[2]; y1 = out[3];
}

// H0 alone, bit-identical to the h0 of hankel01_ld (same sums in the same order, same
// loop exits): the patch sums of the correction need no H1.
static void series0(ld z, ld& j0, ld& y0) {
    const SeriesTables& T = series_tables();
    ld q = z * z / 4;
    ld t0 = 1, t1 = 1;
    ld s0 = 1, a0 = 0;
    for (int k = 1; k <= 40; ++k) {
        t0 *= -q * T.rk2[k];
        t1 *= -q * T.rkk1[k];        // only for the stopping test shared with series01
        s0 += t0;
        a0 += T.hk[k] * t0;
        if (std::fabs(t0) < 1e-24L && std::fabs(t1) < 1e-24L) break;
    }
    ld L = std::log(z / 2) + EG_L;
    j0 = s0;
    y0 = (2 / PI_L) * (L * j0 - a0);
}

static void miller0(ld z, ld& j0, ld& y0) {
    int nstart = 2 * ((int)(z + 56) / 2);
    ld J[96];
    for (int i = 0; i < nstart + 2; ++i) J[i] = 0.0L;
    J[nstart] = 1e-300L;
    for (int n = nstart; n >= 1; --n) {
        J[n - 1] = (2.0L * n / z) * J[n] - J[n + 1];
        if (std::fabs(J[n - 1]) > 1e300L)
            for (int i = n - 1; i <= nstart; ++i) J[i] *= 1e-300L;
    }
    ld norm = J[0];
    for (int k = 2; k <= nstart; k += 2) norm += 2 * J[k];
    for (int i = 0; i < nstart + 2; ++i) J[i] /= norm;
    ld s0 = 0;
    for (int k = 1; 2 * k + 1 <= nstart + 1; ++k) {
        ld sg = (k % 2) ? -1.0L : 1.0L;
        s0 += sg * J[2 * k] / k;
    }
    ld L = std::log(z / 2) + EG_L;
    j0 = J[0];
    y0 = (2 / PI_L) * (L * j0 - 2 * s0);
}

static void asym0(ld z, ld& j0, ld& y0) {
    ld c = std::cos(z), s = std::sin(z);
    ld r2 = std::sqrt(0.5L);
    ld amp = std::sqrt(2 / (PI_L * z));
    ld P = 1, Q = 0, term = 1;
    for (int k = 1; k < 100; ++k) {
        term *= (0.0L - (ld)(2 * k - 1) * (2 * k - 1)) / (k * 8 * z);
        if (k % 2) Q += (((k - 1) / 2) % 2 ? -term : term);
        else       P += ((k / 2) % 2 ? -term : term);
        if (std::fabs(term) < 1e-22L) break;
    }
    ld cc = r2 * (c + s), ss = r2 * (s - c);
    j0 = amp * (P * cc - Q * ss);
    y0 = amp * (P * ss + Q * cc);
}

static cld hankel0_ld(ld z) {
    ld j0, y0;
    if (z <= 6) series0(z, j0, y0);
    else if (z < 30) miller0(z, j0, y0);
    else asym0(z, j0, y0);
    return cld(j0, y0);
}

void hankel01_ld(ld z, cld& h0, cld& h1) {
    ld j0, j1, y0, y1;
    if (z <= 6) series01(z, j0, j1, y0, y1);
    else if (z < 30) miller01(z, j0, j1, y0, y1);
    else asym01(z, j0, j1, y0, y1);
    h0 = cld(j0, y0);
    h1 = cld(j1, y1);
}

// ---------------------------------------------------------------- polynomials
// Scaled monomials s1^a s2^b, a + b <= 4, ordered by degree then by b.
struct Mono { int a, b; };
static const std::array<Mono, 15> MONO = {{{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}, {3, 0}, {2, 1},
                                           {1, 2}, {0, 3}, {4, 0}, {3, 1}, {2, 2}, {1, 3}, {0, 4}}};

static int mono_index(int a, int b) {
    for (int i = 0; i < 15; ++i) if (MONO[i].a == a && MONO[i].b == b) return i;
    return -1;
}

static void mono_eval(ld s1, ld s2, ld* m, ld* g1, ld* g2, ld invh) {
    ld p1[5] = {1, s1, s1 * s1, s1 * s1 * s1, s1 * s1 * s1 * s1};
    ld p2[5] = {1, s2, s2 * s2, s2 * s2 * s2, s2 * s2 * s2 * s2};
    for (int i = 0; i < 15; ++i) {
        int a = MONO[i].a, b = MONO[i].b;
        m[i] = p1[a] * p2[b];
        if (g1) {
            g1[i] = a ? a * p1[a - 1] * p2[b] * invh : 0;
            g2[i] = b ? b * p1[a] * p2[b - 1] * invh : 0;
        }
    }
}

// Gauss-Jordan inverse with partial pivoting (n x n, row-major), false if singular.
static bool invert_ld(ld* A, ld* Ainv, int n) {
    std::vector<ld> M(n * 2 * n);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            M[r * 2 * n + c] = c < n ? A[r * n + c] : (c - n == r ? 1 : 0);
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(M[r * 2 * n + c]) > std::fabs(M[p * 2 * n + c])) p = r;
        if (M[p * 2 * n + c] == 0) return false;
        if (p != c)
            for (int k = 0; k < 2 * n; ++k) std::swap(M[p * 2 * n + k], M[c * 2 * n + k]);
        ld piv = M[c * 2 * n + c];
        for (int k = 0; k < 2 * n; ++k) M[c * 2 * n + k] /= piv;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            ld f = M[r * 2 * n + c];
            if (f == 0) continue;
            for (int k = 0; k < 2 * n; ++k) M[r * 2 * n + k] -= f * M[c * 2 * n + k];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = M[r * 2 * n + n + c];
    return true;
}

// ---------------------------------------------------------------- quadrature
struct GL32 {
    ld x[32], w[32];   // on [0, 1]
    GL32() {
        const int n = 32;
        for (int i = 0; i < n; ++i) {
            ld t = std::cos(PI_L * (i + 0.75L) / (n + 0.5L));
            for (int it = 0; it < 100; ++it) {
                ld p0 = 1, p1 = t;
                for (int m = 2; m <= n; ++m) { ld p2 = ((2 * m - 1) * t * p1 - (m - 1) * p0) / m; p0 = p1; p1 = p2; }
                ld dp = n * (t * p1 - p0) / (t * t - 1);
                ld dt = p1 / dp;
                t -= dt;
                if (std::fabs(dt) < 1e-21L) break;
            }
            ld p0 = 1, p1 = t;
            for (int m = 2; m <= n; ++m) { ld p2 = ((2 * m - 1) * t * p1 - (m - 1) * p0) / m; p0 = p1; p1 = p2; }
            ld dp = n * (t * p1 - p0) / (t * t - 1);
            x[i] = (t + 1) / 2;
            w[i] = 1 / ((1 - t * t) * dp * dp);      // 2 / (...) halved for [0, 1]
        }
    }
};
static const GL32& gl32() { static GL32 g; return g; }

struct Edge {                     // one oriented edge of an element
    ld ax, ay, bx, by;            // straight: endpoints
    bool curved;
    ld cx, cy, R, a, m, phi, t0, t1;
};

static inline void edge_point(const Edge& e, ld t, ld& x, ld& y, ld& dx, ld& dy) {
    if (!e.curved) {
        x = e.ax + t * (e.bx - e.ax);
        y = e.ay + t * (e.by - e.ay);
        dx = e.bx - e.ax;
        dy = e.by - e.ay;
        return;
    }
    ld th = e.t0 + t * (e.t1 - e.t0);
    ld ang = e.m * th + e.phi;
    ld r = e.R * (1 + e.a * std::cos(ang));
    ld dr = -e.R * e.a * e.m * std::sin(ang);
    ld c = std::cos(th), s = std::sin(th);
    x = e.cx + r * c;
    y = e.cy + r * s;
    dx = (dr * c - r * s) * (e.t1 - e.t0);
    dy = (dr * s + r * c) * (e.t1 - e.t0);
}

static Edge make_edge(const HostMesh& M, int t, int e) {
    Edge E{};
    int va = M.tri[3 * t + e], vb = M.tri[3 * t + (e + 1) % 3];
    E.ax = M.vxy[2 * va]; E.ay = M.vxy[2 * va + 1];
    E.bx = M.vxy[2 * vb]; E.by = M.vxy[2 * vb + 1];
    int c = M.ecurve[3 * t + e];
    E.curved = c >= 0;
    if (E.curved) {
        const double* C = &M.curves[6 * c];
        E.cx = C[0]; E.cy = C[1]; E.R = C[2]; E.a = C[3]; E.m = C[4]; E.phi = C[5];
        E.t0 = M.etheta[6 * t + 2 * e]; E.t1 = M.etheta[6 * t + 2 * e + 1];
    }
    return E;
}

struct PolyCtx {                  // one interpolation element
    ld cx, cy, h, invh;
    ld C[15 * 15];                // L_q = sum_a mono_a C[a][q]
    ld Phi[15 * 15];              // Phi_q = sum_a mono_a Phi[a][q]
};

static bool make_poly(const HostMesh& M, int tau, ld k, PolyCtx& P) {
    const int* v = &M.tri[3 * tau];
    ld x0 = M.vxy[2 * v[0]], y0 = M.vxy[2 * v[0] + 1];
    ld x1 = M.vxy[2 * v[1]], y1 = M.vxy[2 * v[1] + 1];
    ld x2 = M.vxy[2 * v[2]], y2 = M.vxy[2 * v[2] + 1];
    P.cx = ((x0 + x1) + x2) / 3;
    P.cy = ((y0 + y1) + y2) / 3;
    ld h2 = std::max({(x0 - x1) * (x0 - x1) + (y0 - y1) * (y0 - y1), (x1 - x2) * (x1 - x2) + (y1 - y2) * (y1 - y2),
                      (x2 - x0) * (x2 - x0) + (y2 - y0) * (y2 - y0)});
    P.h = std::sqrt(h2);
    P.invh = 1 / P.h;
    ld V[225], m[15];
    for (int q = 0; q < 15; ++q) {
        int j = tau * NQ_ELEM + q;
        mono_eval((M.nodes[2 * j] - P.cx) * P.invh, (M.nodes[2 * j + 1] - P.cy) * P.invh, m, nullptr, nullptr, P.invh);
        for (int a = 0; a < 15; ++a) V[q * 15 + a] = m[a];      // V[q][a]
    }
    if (!invert_ld(V, P.C, 15)) return false;                    // C[a][q]
    // Laplacian on coefficient vectors: lap(mono(a,b)) = (a(a-1) mono(a-2,b) + b(b-1) mono(a,b-2)) / h^2
    ld lap1[225], lap2[225];
    auto apply_lap = [&](const ld* src, ld* dst) {
        for (int i = 0; i < 225; ++i) dst[i] = 0;
        for (int a = 0; a < 15; ++a) {
            int ea = MONO[a].a, eb = MONO[a].b;
            for (int q = 0; q < 15; ++q) {
                ld c = src[a * 15 + q];
                if (c == 0) continue;
                if (ea >= 2) dst[mono_index(ea - 2, eb) * 15 + q] += ea * (ea - 1) * c * P.invh * P.invh;
                if (eb >= 2) dst[mono_index(ea, eb - 2) * 15 + q] += eb * (eb - 1) * c * P.invh * P.invh;
            }
        }
    };
    apply_lap(P.C, lap1);
    apply_lap(lap1, lap2);
    ld k2 = k * k;
    for (int i = 0; i < 225; ++i) P.Phi[i] = P.C[i] / k2 - lap1[i] / (k2 * k2) + lap2[i] / (k2 * k2 * k2);
    return true;
}

// Accumulate, over the GL32 points of one panel, the monomial moments
// Mo[a] = sum wt (G d(mono_a)/dn - mono_a dG/dn); E = Phi^T Mo afterwards.
static void panel_integral(const Edge& e, ld ta, ld tb, ld xj, ld yj, ld k, const PolyCtx& P, cld* Mo) {
    const GL32& g = gl32();
    ld m[15], g1[15], g2[15];
    for (int i = 0; i < 32; ++i) {
        ld t = ta + (tb - ta) * g.x[i];
        ld wt = (tb - ta) * g.w[i];
        ld x, y, dx, dy;
        edge_point(e, t, x, y, dx, dy);
        ld nx = dy, ny = -dx;                         // outward normal times |y'|
        ld rx = x - xj, ry = y - yj;
        ld r = std::sqrt(rx * rx + ry * ry);
        cld h0, h1;
        hankel01_ld(k * r, h0, h1);
        cld G = cld(0, 0.25L) * h0;
        cld dGdn = cld(0, 0.25L) * (-k) * h1 * ((rx * nx + ry * ny) / r);
        mono_eval((x - P.cx) * P.invh, (y - P.cy) * P.invh, m, g1, g2, P.invh);
        cld Gw = wt * G, Dw = wt * dGdn;
        for (int a = 0; a < 15; ++a) Mo[a] += Gw * (g1[a] * nx + g2[a] * ny) - Dw * m[a];
    }
}

// Dyadic refinement of the parameter interval [0, 1] of an edge until every panel is
// shorter than 3/4 of its distance to the target (the panels of the boundary rule).
static void edge_panels(const Edge& e, ld xj, ld yj, std::vector<std::pair<ld, ld>>& out) {
    struct Pan { ld a, b; int depth; };
    std::vector<Pan> stack{{0, 1, 0}};
    while (!stack.empty()) {
        Pan p = stack.back();
        stack.pop_back();
        ld xa, ya, xm, ym, xb, yb, d1, d2;
        edge_point(e, p.a, xa, ya, d1, d2);
        edge_point(e, (p.a + p.b) / 2, xm, ym, d1, d2);
        edge_point(e, p.b, xb, yb, d1, d2);
        ld L = std::hypot(xm - xa, ym - ya) + std::hypot(xb - xm, yb - ym);
        ld dist = std::min({std::hypot(xa - xj, ya - yj), std::hypot(xm - xj, ym - yj), std::hypot(xb - xj, yb - yj)});
        if (L > 0.75L * dist && p.depth < 60) {
            ld mid = (p.a + p.b) / 2;
            stack.push_back({p.a, mid, p.depth + 1});
            stack.push_back({mid, p.b, p.depth + 1});
        } else {
            out.push_back({p.a, p.b});
        }
    }
}

static void edge_integral(const Edge& e, ld xj, ld yj, ld k, const PolyCtx& P, cld* Mo) {
    std::vector<std::pair<ld, ld>> pans;
    edge_panels(e, xj, yj, pans);
    for (const auto& p : pans) panel_integral(e, p.first, p.second, xj, yj, k, P, Mo);
}

// Edges met once among the patch elements, as (element, local edge), in a fixed order.
static void patch_boundary(const HostMesh& M, const std::vector<int>& patch, std::vector<std::array<int, 2>>& edges) {
    std::vector<std::array<int, 4>> keys;   // (min v, max v, element, edge)
    keys.reserve(patch.size() * 3);
    for (int t : patch)
        for (int e = 0; e < 3; ++e) {
            int a = M.tri[3 * t + e], b = M.tri[3 * t + (e + 1) % 3];
            keys.push_back({std::min(a, b), std::max(a, b), t, e});
        }
    std::sort(keys.begin(), keys.end());
    for (size_t i = 0; i < keys.size();) {
        size_t r = i + 1;
        while (r < keys.size() && keys[r][0] == keys[i][0] && keys[r][1] == keys[i][1]) ++r;
        if (r - i == 1) edges.push_back({keys[i][2], keys[i][3]});
        i = r;
    }
}

// dV_j,(15 nodes of tau) for the given patch; adds 15 entries to (cols, vals).
static bool correction_block(const HostMesh& M, int j, ld k, const std::vector<int>& patch, int tau, bool own,
                             std::vector<int32_t>& cols, std::vector<std::complex<double>>& vals) {
    PolyCtx P;
    if (!make_poly(M, tau, k, P)) return false;
    ld xj = M.nodes[2 * j], yj = M.nodes[2 * j + 1];
    cld E[15], N[15], Mo[15], Mn[15];
    for (int q = 0; q < 15; ++q) { E[q] = 0; N[q] = 0; Mo[q] = 0; Mn[q] = 0; }
    // boundary edges of the patch: edges met once among the patch elements
    std::vector<std::array<int, 2>> bedges;
    patch_boundary(M, patch, bedges);
    for (const auto& be : bedges) edge_integral(make_edge(M, be[0], be[1]), xj, yj, k, P, Mo);
    for (int q = 0; q < 15; ++q)
        for (int a = 0; a < 15; ++a) E[q] += P.Phi[a * 15 + q] * Mo[a];
    ld m[15];
    if (own) {
        mono_eval((xj - P.cx) * P.invh, (yj - P.cy) * P.invh, m, nullptr, nullptr, P.invh);
        for (int q = 0; q < 15; ++q) {
            ld phi = 0;
            for (int a = 0; a < 15; ++a) phi += m[a] * P.Phi[a * 15 + q];
            E[q] -= phi;
        }
    }
    for (int t : patch)
        for (int qq = 0; qq < NQ_ELEM; ++qq) {
            int n = t * NQ_ELEM + qq;
            if (n == j) continue;
            ld yx = M.nodes[2 * n], yy = M.nodes[2 * n + 1];
            ld r = std::sqrt((yx - xj) * (yx - xj) + (yy - yj) * (yy - yj));
            cld h0 = hankel0_ld(k * r);
            cld Gw = cld(0, 0.25L) * h0 * (ld)M.w[n];
            mono_eval((yx - P.cx) * P.invh, (yy - P.cy) * P.invh, m, nullptr, nullptr, P.invh);
            for (int a = 0; a < 15; ++a) Mn[a] += Gw * m[a];
        }
    for (int q = 0; q < 15; ++q)
        for (int a = 0; a < 15; ++a) N[q] += P.C[a * 15 + q] * Mn[a];
    for (int q = 0; q < 15; ++q) {
        cols.push_back(tau * NQ_ELEM + q);
        cld d = E[q] - N[q];
        vals.push_back(std::complex<double>((double)d.real(), (double)d.imag()));
    }
    return true;
}

#pragma GCC push_options
#pragma GCC optimize("fp-contract=off")
// Element centroid and squared size, computed exactly as documented (float64, no FMA).
static void element_geometry(const HostMesh& M, std::vector<double>& cen, std::vector<double>& h2) {
    cen.resize(2 * M.nt);
    h2.resize(M.nt);
    for (int t = 0; t < M.nt; ++t) {
        const int* v = &M.tri[3 * t];
        double x0 = M.vxy[2 * v[0]], y0 = M.vxy[2 * v[0] + 1];
        double x1 = M.vxy[2 * v[1]], y1 = M.vxy[2 * v[1] + 1];
        double x2 = M.vxy[2 * v[2]], y2 = M.vxy[2 * v[2] + 1];
        cen[2 * t] = ((x0 + x1) + x2) / 3.0;
        cen[2 * t + 1] = ((y0 + y1) + y2) / 3.0;
        double a = (x0 - x1) * (x0 - x1) + (y0 - y1) * (y0 - y1);
        double b = (x1 - x2) * (x1 - x2) + (y1 - y2) * (y1 - y2);
        double c = (x2 - x0) * (x2 - x0) + (y2 - y0) * (y2 - y0);
        h2[t] = std::max(std::max(a, b), c);
    }
}

static inline double dist2(double ax, double ay, double bx, double by) {
    double dx = ax - bx, dy = ay - by;
    return dx * dx + dy * dy;
}
#pragma GCC pop_options

// Patches of every target: element centroids bucketed on a grid of cells no smaller
// than the largest patch radius, so a patch lies in the 3 x 3 cells around its target.
struct PatchBlock {
    std::vector<int> elems;       // sorted element ids of the patch in one subdomain
    int tau;                      // interpolation element (own element, or the nearest one)
    bool own;                     // the target's own subdomain
};

class PatchFinder {
  public:
    PatchFinder(const HostMesh& M, double kappa) : M_(M), kappa_(kappa) {
        element_geometry(M, cen_, h2_);
        for (int d : M.dom) ndom_ = std::max(ndom_, d + 1);
        double rmax = 0;
        xmin_ = ymin_ = 1e300;
        double xmax = -1e300, ymax = -1e300;
        for (int t = 0; t < M.nt; ++t) {
            rmax = std::max(rmax, kappa * std::sqrt(h2_[t]));
            xmin_ = std::min(xmin_, cen_[2 * t]); xmax = std::max(xmax, cen_[2 * t]);
            ymin_ = std::min(ymin_, cen_[2 * t + 1]); ymax = std::max(ymax, cen_[2 * t + 1]);
        }
        cell_ = std::max(rmax, 1e-12) * 1.0000001;
        gx_ = std::max(1, (int)std::ceil((xmax - xmin_) / cell_) + 1);
        gy_ = std::max(1, (int)std::ceil((ymax - ymin_) / cell_) + 1);
        bucket_.resize((size_t)gx_ * gy_);
        for (int t = 0; t < M.nt; ++t) {
            int bx = std::min(gx_ - 1, (int)((cen_[2 * t] - xmin_) / cell_));
            int by = std::min(gy_ - 1, (int)((cen_[2 * t + 1] - ymin_) / cell_));
            bucket_[(size_t)by * gx_ + bx].push_back(t);
        }
    }

    // Blocks of target j in subdomain order (patch rule as documented at the top).
    void blocks(int j, std::vector<PatchBlock>& out) const {
        out.clear();
        const int tau = j / NQ_ELEM, l = M_.dom[tau];
        const double xj = M_.nodes[2 * j], yj = M_.nodes[2 * j + 1];
        const double thr = kappa_ * kappa_ * h2_[tau];
        const int bx = std::min(gx_ - 1, std::max(0, (int)((xj - xmin_) / cell_)));
        const int by = std::min(gy_ - 1, std::max(0, (int)((yj - ymin_) / cell_)));
        std::vector<std::vector<int>> patch(ndom_);
        for (int cy = std::max(0, by - 1); cy <= std::min(gy_ - 1, by + 1); ++cy)
            for (int cx = std::max(0, bx - 1); cx <= std::min(gx_ - 1, bx + 1); ++cx)
                for (int t : bucket_[(size_t)cy * gx_ + cx])
                    if (dist2(cen_[2 * t], cen_[2 * t + 1], xj, yj) < thr) patch[M_.dom[t]].push_back(t);
        for (int d = 0; d < ndom_; ++d) {
            auto& P = patch[d];
            std::sort(P.begin(), P.end());
            int interp;
            if (d == l) {
                if (!std::binary_search(P.begin(), P.end(), tau)) P.insert(std::lower_bound(P.begin(), P.end(), tau), tau);
                interp = tau;
            } else {
                if (P.empty()) continue;
                interp = P[0];
                double best = dist2(cen_[2 * P[0]], cen_[2 * P[0] + 1], xj, yj);
                for (int t : P) {
                    double d2 = dist2(cen_[2 * t], cen_[2 * t + 1], xj, yj);
                    if (d2 < best) { best = d2; interp = t; }
                }
            }
            out.push_back(PatchBlock{std::move(P), interp, d == l});
        }
    }

  private:
    const HostMesh& M_;
    double kappa_;
    std::vector<double> cen_, h2_;
    int ndom_ = 0, gx_ = 1, gy_ = 1;
    double xmin_ = 0, ymin_ = 0, cell_ = 1;
    std::vector<std::vector<int>> bucket_;
};

std::string build_correction(const HostMesh& M, double k, double kappa, CsrC& out) {
    PatchFinder finder(M, kappa);
    const int nq = M.nq;
    std::vector<std::vector<int32_t>> rcols(nq);
    std::vector<std::vector<std::complex<double>>> rvals(nq);
    int failed = -1;
    const ld kl = k;
#pragma omp parallel for schedule(dynamic, 16)
    for (int j = 0; j < nq; ++j) {
        std::vector<PatchBlock> blk;
        finder.blocks(j, blk);
        for (const auto& B : blk)
            if (!correction_block(M, j, kl, B.elems, B.tau, B.own, rcols[j], rvals[j])) {
#pragma omp critical
                failed = j;
            }
    }
    if (failed >= 0) return "singular interpolation matrix for target " + std::to_string(failed);
    out.rowptr.assign(nq + 1, 0);
    for (int j = 0; j < nq; ++j) out.rowptr[j + 1] = out.rowptr[j] + (int64_t)rcols[j].size();
    out.cols.resize(out.rowptr[nq]);
    out.vals.resize(out.rowptr[nq]);
    for (int j = 0; j < nq; ++j) {
        std::copy(rcols[j].begin(), rcols[j].end(), out.cols.begin() + out.rowptr[j]);
        std::copy(rvals[j].begin(), rvals[j].end(), out.vals.begin() + out.rowptr[j]);
    }
    return "";
}

// ---------------------------------------------------------------- plan of the device build
std::string plan_correction(const HostMesh& M, double kappa, CorrPlan& P) {
    PatchFinder finder(M, kappa);
    const int nq = M.nq;
    struct Local {
        std::vector<int32_t> tau, nelem, npan, elems, pedge;
        std::vector<int8_t> own;
        std::vector<long double> pa, pb;
    };
    std::vector<Local> per(nq);
#pragma omp parallel for schedule(dynamic, 16)
    for (int j = 0; j < nq; ++j) {
        std::vector<PatchBlock> blk;
        finder.blocks(j, blk);
        Local& L = per[j];
        const ld xj = M.nodes[2 * j], yj = M.nodes[2 * j + 1];
        for (const auto& B : blk) {
            L.tau.push_back(B.tau);
            L.own.push_back(B.own ? 1 : 0);
            L.nelem.push_back((int32_t)B.elems.size());
            L.elems.insert(L.elems.end(), B.elems.begin(), B.elems.end());
            std::vector<std::array<int, 2>> bedges;
            patch_boundary(M, B.elems, bedges);
            int np = 0;
            for (const auto& be : bedges) {
                std::vector<std::pair<ld, ld>> pans;
                edge_panels(make_edge(M, be[0], be[1]), xj, yj, pans);
                for (const auto& p : pans) {
                    L.pedge.push_back(3 * be[0] + be[1]);
                    L.pa.push_back(p.first);
                    L.pb.push_back(p.second);
                    ++np;
                }
            }
            L.npan.push_back(np);
        }
    }
    P = CorrPlan{};
    P.row_blocks.assign(nq + 1, 0);
    for (int j = 0; j < nq; ++j) P.row_blocks[j + 1] = P.row_blocks[j] + (int64_t)per[j].tau.size();
    const int64_t nb = P.row_blocks[nq];
    P.target.resize(nb); P.tau.resize(nb); P.own.resize(nb);
    P.elem_off.assign(nb + 1, 0);
    P.pan_off.assign(nb + 1, 0);
    for (int j = 0; j < nq; ++j) {
        const Local& L = per[j];
        int64_t b0 = P.row_blocks[j];
        for (size_t i = 0; i < L.tau.size(); ++i) {
            P.target[b0 + i] = j;
            P.tau[b0 + i] = L.tau[i];
            P.own[b0 + i] = L.own[i];
            P.elem_off[b0 + i + 1] = L.nelem[i];
            P.pan_off[b0 + i + 1] = L.npan[i];
        }
    }
    for (int64_t b = 0; b < nb; ++b) {
        P.elem_off[b + 1] += P.elem_off[b];
        P.pan_off[b + 1] += P.pan_off[b];
    }
    P.elems.reserve(P.elem_off[nb]);
    P.pan_edge.reserve(P.pan_off[nb]);
    P.pan_a.reserve(P.pan_off[nb]);
    P.pan_b.reserve(P.pan_off[nb]);
    for (int j = 0; j < nq; ++j) {
        const Local& L = per[j];
        P.elems.insert(P.elems.end(), L.elems.begin(), L.elems.end());
        P.pan_edge.insert(P.pan_edge.end(), L.pedge.begin(), L.pedge.end());
        P.pan_a.insert(P.pan_a.end(), L.pa.begin(), L.pa.end());
        P.pan_b.insert(P.pan_b.end(), L.pb.begin(), L.pb.end());
    }
    return "";
}

bool poly_context(const HostMesh& M, int tau, double k, long double* c3, long double* C, long double* Phi) {
    PolyCtx P;
    if (!make_poly(M, tau, k, P)) return false;
    c3[0] = P.cx; c3[1] = P.cy; c3[2] = P.invh;
    std::copy(P.C, P.C + 225, C);
    std::copy(P.Phi, P.Phi + 225, Phi);
    return true;
}

bool correction_block_host(const HostMesh& M, int j, double k, const std::vector<int>& patch, int tau, bool own,
                           std::complex<double>* out15) {
    std::vector<int32_t> cols;
    std::vector<std::complex<double>> vals;
    if (!correction_block(M, j, (ld)k, patch, tau, own, cols, vals)) return false;
    std::copy(vals.begin(), vals.end(), out15);
    return true;
}

void gl32_unit(long double* x, long double* w) {
    const GL32& g = gl32();
    std::copy(g.x, g.x + 32, x);
    std::copy(g.w, g.w + 32, w);
}

// ---------------------------------------------------------------- H0 table
// Chebyshev interpolation of H0(k sqrt(t)) at ncoef points per cell, converted
// to monomials in u; each octave is refined (2^m cells, m >= 3) until the
// interpolant matches the long-double routine to tol (relative) at 33 points
// per cell.
std::string build_h0_table(double k, double t_lo, double t_hi, H0Table& T, int ncoef, double tol) {
    if (!(t_lo > 0) || !(t_hi > t_lo)) return "bad table range";
    if (ncoef < 2 || ncoef > 16) return "bad table degree";
    const int NC = ncoef;
    int e_lo, e_hi;
    std::frexp(t_lo, &e_lo);          // t in [2^(e-1), 2^e)
    std::frexp(t_hi, &e_hi);
    T.b_lo = e_lo - 1 + 1023;
    T.noct = e_hi - e_lo + 1;
    T.oct_base.assign(T.noct, 0);
    T.oct_shift.assign(T.noct, 0);
    T.mid.clear(); T.inv_hw.clear(); T.coef.clear();
    T.max_rel_err = 0;
    // monomial coefficients of T_n(u), n < NC
    std::vector<std::vector<ld>> cheb(NC, std::vector<ld>(NC, 0));
    std::vector<ld> un(NC);
    cheb[0][0] = 1;
    if (NC > 1) cheb[1][1] = 1;
    for (int n = 2; n < NC; ++n)
        for (int j = 0; j < NC; ++j)
            cheb[n][j] = (j > 0 ? 2 * cheb[n - 1][j - 1] : 0) - cheb[n - 2][j];
    for (int i = 0; i < NC; ++i) un[i] = std::cos(PI_L * (i + 0.5L) / NC);
    const ld kl = k;
    for (int o = 0; o < T.noct; ++o) {
        ld a = std::ldexp(1.0L, e_lo - 1 + o), b = 2 * a;
        std::vector<double> bm, bi;
        std::vector<std::complex<double>> bc;
        int m = 3;
        for (;; ++m) {
            int M = 1 << m;
            bm.assign(M, 0); bi.assign(M, 0); bc.assign((size_t)M * NC, 0);
            double worst = 0;
            for (int c = 0; c < M; ++c) {
                ld lo = a + (b - a) * c / M, hi = a + (b - a) * (c + 1) / M;
                ld mid = (lo + hi) / 2, hw = (hi - lo) / 2;
                std::vector<cld> f(NC), cc(NC), mono(NC);
                for (int i = 0; i < NC; ++i) {
                    cld h0, h1;
                    hankel01_ld(kl * std::sqrt(mid + hw * un[i]), h0, h1);
                    f[i] = h0;
                }
                for (int n = 0; n < NC; ++n) {
                    cld acc = 0;
                    for (int i = 0; i < NC; ++i) acc += f[i] * std::cos(n * PI_L * (i + 0.5L) / NC);
                    cc[n] = acc * (n == 0 ? 1.0L : 2.0L) / (ld)NC;
                }
                for (int j = 0; j < NC; ++j) {
                    mono[j] = 0;
                    for (int n = 0; n < NC; ++n) mono[j] += cc[n] * cheb[n][j];
                }
                for (int q = 0; q <= 32; ++q) {
                    ld u = -1 + 2.0L * q / 32;
                    cld p = 0;
                    for (int j = NC - 1; j >= 0; --j) p = p * u + mono[j];
                    cld h0, h1;
                    hankel01_ld(kl * std::sqrt(mid + hw * u), h0, h1);
                    worst = std::max(worst, (double)(std::abs(p - h0) / std::abs(h0)));
                }
                bm[c] = (double)mid;
                bi[c] = (double)(1 / hw);
                for (int j = 0; j < NC; ++j)
                    bc[(size_t)c * NC + j] = std::complex<double>((double)mono[j].real(), (double)mono[j].imag());
            }
            if (worst <= tol || m >= 12) {
                T.max_rel_err = std::max(T.max_rel_err, worst);
                break;
            }
        }
        T.oct_base[o] = (int)T.mid.size();
        T.oct_shift[o] = 20 - m;
        T.mid.insert(T.mid.end(), bm.begin(), bm.end());
        T.inv_hw.insert(T.inv_hw.end(), bi.begin(), bi.end());
        T.coef.insert(T.coef.end(), bc.begin(), bc.end());
    }
    return "";
}

// ---------------------------------------------------------------- grid
static std::complex<double> vc_entry(ld k, ld h, int da, int db) {
    if (da == 0 && db == 0) {
        ld a = h / std::sqrt(PI_L);
        cld h0, h1;
        hankel01_ld(k * a, h0, h1);
        cld v = cld(0, PI_L) * a * h1 / (2 * k) - 1 / (k * k);
        return std::complex<double>((double)v.real(), (double)v.imag());
    }
    ld r = h * std::sqrt((ld)da * da + (ld)db * db);
    cld h0, h1;
    hankel01_ld(k * r, h0, h1);
    cld v = cld(0, 0.25L) * h0 * h * h;
    return std::complex<double>((double)v.real(), (double)v.imag());
}

// Hermitian 9 x 9 Jacobi eigen-solver (long double); returns the eigenvector of the
// smallest eigenvalue in vec.
static void smallest_eigvec(std::vector<cld>& A, int n, std::vector<cld>& vec) {
    std::vector<cld> Vm(n * n, cld(0, 0));
    for (int i = 0; i < n; ++i) Vm[i * n + i] = 1;
    for (int sweep = 0; sweep < 100; ++sweep) {
        ld off = 0, tot = 0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                ld a2 = std::norm(A[p * n + q]);
                tot += a2;
                if (p != q) off += a2;
            }
        if (off <= 1e-38L * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                cld apq = A[p * n + q];
                ld aabs = std::abs(apq);
                if (aabs == 0) continue;
                ld app = A[p * n + p].real(), aqq = A[q * n + q].real();
                // rotation zeroing A[p][q]: unitary [[c, -s e^{i phi}], [s e^{-i phi}, c]]
                cld ph = apq / aabs;
                ld theta = 0.5L * std::atan2(2 * aabs, aqq - app);
                ld c = std::cos(theta), s = std::sin(theta);
                // columns p, q
                for (int r = 0; r < n; ++r) {
                    cld arp = A[r * n + p], arq = A[r * n + q];
                    A[r * n + p] = c * arp - s * std::conj(ph) * arq;
                    A[r * n + q] = s * ph * arp + c * arq;
                    cld vrp = Vm[r * n + p], vrq = Vm[r * n + q];
                    Vm[r * n + p] = c * vrp - s * std::conj(ph) * vrq;
                    Vm[r * n + q] = s * ph * vrp + c * vrq;
                }
                // rows p, q
                for (int r = 0; r < n; ++r) {
                    cld apr = A[p * n + r], aqr = A[q * n + r];
                    A[p * n + r] = c * apr - s * ph * aqr;
                    A[q * n + r] = s * std::conj(ph) * apr + c * aqr;
                }
            }
    }
    int best = 0;
    for (int i = 1; i < n; ++i) if (A[i * n + i].real() < A[best * n + best].real()) best = i;
    vec.resize(n);
    for (int r = 0; r < n; ++r) vec[r] = Vm[r * n + best];
}

// ---------------------------------------------------------------- Approach I transfer
// Element map of the mesh: the affine map of the vertex triangle plus, for an element
// with a curved edge e (vertices i = e, j = e + 1), the edge bubble 4 l_i l_j d(t),
// t = (1 + l_j - l_i) / 2, d(t) = (gamma(theta(t)) - chord(t)) / (4 t (1 - t)), which puts
// that edge on its polar curve and keeps the other two straight.
static void element_point(const HostMesh& M, int t, double xi, double eta, double& x, double& y) {
    const int* v = &M.tri[3 * t];
    const double l[3] = {1.0 - xi - eta, xi, eta};
    x = 0; y = 0;
    for (int a = 0; a < 3; ++a) { x += l[a] * M.vxy[2 * v[a]]; y += l[a] * M.vxy[2 * v[a] + 1]; }
    for (int e = 0; e < 3; ++e) {
        const int c = M.ecurve[3 * t + e];
        if (c < 0) continue;
        const int i = e, j = (e + 1) % 3;
        const double li = l[i], lj = l[j];
        if (li * lj == 0.0) return;
        const double tt = 0.5 * (1.0 + lj - li);
        const double* C = &M.curves[6 * c];
        const double th = M.etheta[6 * t + 2 * e] + tt * (M.etheta[6 * t + 2 * e + 1] - M.etheta[6 * t + 2 * e]);
        const double r = C[2] * (1.0 + C[3] * std::cos(C[4] * th + C[5]));
        const double gx = C[0] + r * std::cos(th), gy = C[1] + r * std::sin(th);
        const double den = 4.0 * tt * (1.0 - tt);
        const double dx = (gx - ((1 - tt) * M.vxy[2 * v[i]] + tt * M.vxy[2 * v[j]])) / den;
        const double dy = (gy - ((1 - tt) * M.vxy[2 * v[i] + 1] + tt * M.vxy[2 * v[j] + 1])) / den;
        x += 4.0 * li * lj * dx;
        y += 4.0 * li * lj * dy;
        return;
    }
}

// Element owning each grid node (-1: none).  A node is in element t when Newton's method
// on t's map (central-difference Jacobian, started from the affine inverse) lands in the
// closed reference triangle (tolerance 1e-12); the lowest such element index wins.
static void locate_grid_nodes(const HostMesh& M, const GridSetup& G, std::vector<int>& owner) {
    owner.assign((size_t)G.nx * G.ny, -1);
    for (int t = 0; t < M.nt; ++t) {
        const int* v = &M.tri[3 * t];
        double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
        auto grow = [&](double x, double y) {
            xmin = std::min(xmin, x); xmax = std::max(xmax, x); ymin = std::min(ymin, y); ymax = std::max(ymax, y);
        };
        for (int a = 0; a < 3; ++a) grow(M.vxy[2 * v[a]], M.vxy[2 * v[a] + 1]);
        for (int i = 0; i < 32; ++i) {
            const double s_ = (i + 0.5) / 32;
            double x, y;
            element_point(M, t, s_, 0.0, x, y); grow(x, y);
            element_point(M, t, 0.0, s_, x, y); grow(x, y);
            element_point(M, t, 1.0 - s_, s_, x, y); grow(x, y);
        }
        const double pad = 1e-9 * (1.0 + (xmax - xmin) + (ymax - ymin));
        const int a0 = std::max(0, (int)std::ceil((xmin - pad - G.x0) / G.h));
        const int a1 = std::min(G.nx - 1, (int)std::floor((xmax + pad - G.x0) / G.h));
        const int b0 = std::max(0, (int)std::ceil((ymin - pad - G.y0) / G.h));
        const int b1 = std::min(G.ny - 1, (int)std::floor((ymax + pad - G.y0) / G.h));
        const double x0 = M.vxy[2 * v[0]], y0 = M.vxy[2 * v[0] + 1];
        const double A00 = M.vxy[2 * v[1]] - x0, A01 = M.vxy[2 * v[2]] - x0;
        const double A10 = M.vxy[2 * v[1] + 1] - y0, A11 = M.vxy[2 * v[2] + 1] - y0;
        const double det = A00 * A11 - A01 * A10;
        for (int b = b0; b <= b1; ++b)
            for (int a = a0; a <= a1; ++a) {
                const size_t j = a + (size_t)G.nx * b;
                if (owner[j] >= 0) continue;
                const double zx = G.x0 + a * G.h, zy = G.y0 + b * G.h;
                double xi = (A11 * (zx - x0) - A01 * (zy - y0)) / det;
                double eta = (-A10 * (zx - x0) + A00 * (zy - y0)) / det;
                bool ok = true;
                for (int it = 0; it < 40; ++it) {
                    double fx, fy, px, py, mx, my, qx, qy, nx_, ny_;
                    element_point(M, t, xi, eta, fx, fy);
                    const double hd = 1e-7;
                    element_point(M, t, xi + hd, eta, px, py);
                    element_point(M, t, xi - hd, eta, mx, my);
                    element_point(M, t, xi, eta + hd, qx, qy);
                    element_point(M, t, xi, eta - hd, nx_, ny_);
                    const double j00 = (px - mx) / (2 * hd), j10 = (py - my) / (2 * hd);
                    const double j01 = (qx - nx_) / (2 * hd), j11 = (qy - ny_) / (2 * hd);
                    const double dj = j00 * j11 - j01 * j10;
                    const double rx = fx - zx, ry = fy - zy;
                    if (!(std::isfinite(dj) && std::isfinite(rx) && std::isfinite(ry)) || dj == 0.0) { ok = false; break; }
                    const double sx = (j11 * rx - j01 * ry) / dj, sy = (-j10 * rx + j00 * ry) / dj;
                    xi -= sx;
                    eta -= sy;
                    if (std::max(std::fabs(sx), std::fabs(sy)) < 1e-15) break;
                }
                if (ok && xi >= -1e-12 && eta >= -1e-12 && xi + eta <= 1 + 1e-12) owner[j] = t;
            }
    }
}

// Barycentric coordinates of (x, y) in the straight triangle of element t's vertices.
static void bary(const HostMesh& M, int t, double x, double y, double* lam) {
    const int* v = &M.tri[3 * t];
    const double x0 = M.vxy[2 * v[0]], y0 = M.vxy[2 * v[0] + 1];
    const double A00 = M.vxy[2 * v[1]] - x0, A01 = M.vxy[2 * v[2]] - x0;
    const double A10 = M.vxy[2 * v[1] + 1] - y0, A11 = M.vxy[2 * v[2] + 1] - y0;
    const double det = A00 * A11 - A01 * A10;
    lam[1] = (A11 * (x - x0) - A01 * (y - y0)) / det;
    lam[2] = (-A10 * (x - x0) + A00 * (y - y0)) / det;
    lam[0] = 1.0 - lam[1] - lam[2];
}

// Transpose of a gather CSR (rows x ncols) into a gather CSR over the columns.
static void csr_transpose(int nrows, int ncols, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                          const std::vector<double>& cv, std::vector<int64_t>& rpT, std::vector<int32_t>& ciT,
                          std::vector<double>& cvT) {
    rpT.assign(ncols + 1, 0);
    for (int32_t c : ci) rpT[c + 1]++;
    for (int c = 0; c < ncols; ++c) rpT[c + 1] += rpT[c];
    ciT.resize(ci.size());
    cvT.resize(cv.size());
    std::vector<int64_t> fill(rpT.begin(), rpT.end() - 1);
    for (int r = 0; r < nrows; ++r)
        for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
            const int64_t pos = fill[ci[e]]++;
            ciT[pos] = r;
            cvT[pos] = cv[e];
        }
}

std::string build_transfers(const HostMesh& M, const double box[4], int nx, int ny, int approach, GridSetup& G) {
    if (nx < 4 || ny < 4) return "grid needs at least 4 x 4 nodes";
    double hx = (box[1] - box[0]) / (nx - 1), hy = (box[3] - box[2]) / (ny - 1);
    if (!(hx > 0) || std::fabs(hx - hy) > 1e-12 * hx) return "grid step must be equal in x and y";
    G.nx = nx; G.ny = ny; G.x0 = box[0]; G.y0 = box[2]; G.h = hx;
    const int nq = M.nq, nc = nx * ny;
    G.tcq_idx.resize(4 * (size_t)nq);
    G.tcq_w.resize(4 * (size_t)nq);
    std::vector<double> colsum(nc, 0.0);
    for (int q = 0; q < nq; ++q) {
        double yx = M.nodes[2 * q], yy = M.nodes[2 * q + 1];
        if (yx < box[0] || yx > box[1] || yy < box[2] || yy > box[3]) return "quadrature node outside the grid box";
        int a = (int)std::floor((yx - G.x0) / G.h), b = (int)std::floor((yy - G.y0) / G.h);
        a = std::min(std::max(a, 0), nx - 2);
        b = std::min(std::max(b, 0), ny - 2);
        int c = 0;
        for (int db = 0; db < 2; ++db)
            for (int da = 0; da < 2; ++da) {
                double zx = G.x0 + (a + da) * G.h, zy = G.y0 + (b + db) * G.h;
                double psi = (1 - std::fabs(yx - zx) / G.h) * (1 - std::fabs(yy - zy) / G.h);
                int idx = (a + da) + nx * (b + db);
                G.tcq_idx[4 * (size_t)q + c] = idx;
                G.tcq_w[4 * (size_t)q + c] = psi;
                colsum[idx] += psi;
                ++c;
            }
    }
    G.D.resize(nc);
    for (int i = 0; i < nc; ++i) G.D[i] = colsum[i] > 0 ? colsum[i] : 1.0;
    // gather CSR of (T_C^Q)^T over grid rows; Approach II: T_Q^C = D^{-1} (T_C^Q)^T
    G.tcqT_rowptr.assign(nc + 1, 0);
    for (size_t e = 0; e < 4 * (size_t)nq; ++e) G.tcqT_rowptr[G.tcq_idx[e] + 1]++;
    for (int i = 0; i < nc; ++i) G.tcqT_rowptr[i + 1] += G.tcqT_rowptr[i];
    G.tcqT_cols.resize(4 * (size_t)nq);
    G.tcqT_vals.resize(4 * (size_t)nq);
    std::vector<int64_t> fill(G.tcqT_rowptr.begin(), G.tcqT_rowptr.end() - 1);
    for (int q = 0; q < nq; ++q)
        for (int c = 0; c < 4; ++c) {
            int i = G.tcq_idx[4 * (size_t)q + c];
            int64_t pos = fill[i]++;
            G.tcqT_cols[pos] = q;
            G.tcqT_vals[pos] = G.tcq_w[4 * (size_t)q + c];
        }
    if (approach == 2) {
        G.tqc_rowptr = G.tcqT_rowptr;
        G.tqc_cols = G.tcqT_cols;
        G.tqc_vals.resize(G.tcqT_vals.size());
        for (int i = 0; i < nc; ++i)
            for (int64_t e = G.tqc_rowptr[i]; e < G.tqc_rowptr[i + 1]; ++e) G.tqc_vals[e] = G.tcqT_vals[e] / G.D[i];
        G.n_interior = 0;
        for (int i = 0; i < nc; ++i) G.n_interior += colsum[i] > 0;
    } else {
        // Approach I (Eq. T_HC_proj_def): z_j in element t gets
        // T[j, q] = w_q sum_{i, i'} phi_i(z_j) (3 / |t|) [3 delta_ii' - (1 - delta_ii')] phi_i'(y_q)
        std::vector<int> owner;
        locate_grid_nodes(M, G, owner);
        G.tqc_rowptr.assign(nc + 1, 0);
        G.tqc_cols.clear();
        G.tqc_vals.clear();
        G.n_interior = 0;
        for (int j = 0; j < nc; ++j) {
            const int t = owner[j];
            if (t >= 0) {
                ++G.n_interior;
                const int* v = &M.tri[3 * t];
                const double area = 0.5 * std::fabs((M.vxy[2 * v[1]] - M.vxy[2 * v[0]]) * (M.vxy[2 * v[2] + 1] - M.vxy[2 * v[0] + 1]) -
                                                    (M.vxy[2 * v[2]] - M.vxy[2 * v[0]]) * (M.vxy[2 * v[1] + 1] - M.vxy[2 * v[0] + 1]));
                double pz[3];
                bary(M, t, G.x0 + (j % nx) * G.h, G.y0 + (j / nx) * G.h, pz);
                // c_i' = sum_i phi_i(z) Minv_{i i'}
                double cz[3];
                for (int i2 = 0; i2 < 3; ++i2) {
                    double acc = 0;
                    for (int i = 0; i < 3; ++i) acc += pz[i] * (i == i2 ? 3.0 : -1.0);
                    cz[i2] = acc * 3.0 / area;
                }
                for (int q = 0; q < NQ_ELEM; ++q) {
                    const int n = t * NQ_ELEM + q;
                    double pq[3];
                    bary(M, t, M.nodes[2 * n], M.nodes[2 * n + 1], pq);
                    G.tqc_cols.push_back(n);
                    G.tqc_vals.push_back(M.w[n] * (cz[0] * pq[0] + cz[1] * pq[1] + cz[2] * pq[2]));
                }
            }
            G.tqc_rowptr[j + 1] = (int64_t)G.tqc_cols.size();
        }
    }
    csr_transpose(nc, nq, G.tqc_rowptr, G.tqc_cols, G.tqc_vals, G.tqcT_rowptr, G.tqcT_cols, G.tqcT_vals);
    return "";
}

std::string build_grid(const HostMesh& M, double k, const double box[4], int nx, int ny,
                       const std::complex<double>* m_grid, GridSetup& G, int approach) {
    std::string err = build_transfers(M, box, nx, ny, approach, G);
    if (!err.empty()) return err;
    return build_stencil_C(k, box, nx, ny, m_grid, G);
}

void cartesian_kernel_table(double k, double h, int nx, int ny, std::vector<std::complex<double>>& K) {
    K.assign((size_t)nx * ny, 0.0);
#pragma omp parallel for schedule(dynamic, 8)
    for (int b = 0; b < ny; ++b)
        for (int a = 0; a < nx; ++a) K[(size_t)b * nx + a] = vc_entry((ld)k, (ld)h, a, b);
}

std::string build_stencil_C(double k, const double box[4], int nx, int ny, const std::complex<double>* m_grid,
                            GridSetup& G) {
    if (nx < 4 || ny < 4) return "grid needs at least 4 x 4 nodes";
    const double hx = (box[1] - box[0]) / (nx - 1), hy = (box[3] - box[2]) / (ny - 1);
    if (!(hx > 0) || std::fabs(hx - hy) > 1e-12 * hx) return "grid step must be equal in x and y";
    G.nx = nx; G.ny = ny; G.x0 = box[0]; G.y0 = box[2]; G.h = hx;
    const int nc = nx * ny;
    // stencils: per row class c = ca + 3 cb, the truncated neighbourhood N(j) of a
    // representative node (grid centre, middle of an edge, corner), Gram matrix of
    // B = V^(C)(N(j), N(j)^c) against every other grid node, smallest eigenvector
    const ld kl = k, hl = G.h;
    int nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        nthreads = omp_get_num_threads();
    }
#endif
    const int rep_a[3] = {0, nx / 2, nx - 1}, rep_b[3] = {0, ny / 2, ny - 1};
    for (int c = 0; c < 9; ++c) {
        const int ca = rep_a[c % 3], cb = rep_b[c / 3];
        int offs[9], no = 0;
        for (int s = 0; s < 9; ++s) {
            int la = ca + s % 3 - 1, lb = cb + s / 3 - 1;
            if (la >= 0 && la < nx && lb >= 0 && lb < ny) offs[no++] = s;
        }
        std::vector<std::vector<cld>> part(nthreads, std::vector<cld>(81, cld(0, 0)));
#pragma omp parallel for schedule(static)
        for (int l = 0; l < nc; ++l) {
            int la = l % nx, lb = l / nx;
            if (std::abs(la - ca) <= 1 && std::abs(lb - cb) <= 1) continue;
            cld col[9];
            for (int i = 0; i < no; ++i) {
                int da = offs[i] % 3 - 1, db = offs[i] / 3 - 1;
                ld r = hl * std::sqrt((ld)(la - ca - da) * (la - ca - da) + (ld)(lb - cb - db) * (lb - cb - db));
                cld h0, h1;
                hankel01_ld(kl * r, h0, h1);
                col[i] = cld(0, 0.25L) * h0 * hl * hl;
            }
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            for (int p = 0; p < no; ++p)
                for (int q = 0; q < no; ++q) part[tid][p * no + q] += col[p] * std::conj(col[q]);
        }
        std::vector<cld> gram((size_t)no * no, cld(0, 0));
        for (auto& pp : part)
            for (int i = 0; i < no * no; ++i) gram[i] += pp[i];
        std::vector<cld> u;
        smallest_eigvec(gram, no, u);
        // v = conj(u), unit norm; zero at offsets outside the grid
        ld nrm = 0;
        for (auto& x : u) nrm += std::norm(x);
        nrm = std::sqrt(nrm);
        for (int s = 0; s < 9; ++s) G.v[c][s] = 0.0;
        for (int i = 0; i < no; ++i) {
            cld vs = std::conj(u[i]) / nrm;
            G.v[c][offs[i]] = std::complex<double>((double)vs.real(), (double)vs.imag());
        }
    }
    // V^(C) on offsets [-2, 2]^2
    std::complex<double> vcoff[5][5];
    for (int da = -2; da <= 2; ++da)
        for (int db = -2; db <= 2; ++db) vcoff[da + 2][db + 2] = vc_entry(kl, hl, da, db);
    // C = A L^(C) on the 3x3 pattern, every row with the stencil of its class
    G.cband.assign((size_t)ny * 9 * nx, std::complex<double>(0, 0));
    const double k2 = k * k;
    for (int b = 0; b < ny; ++b)
        for (int a = 0; a < nx; ++a) {
            const int cls = (a == 0 ? 0 : (a == nx - 1 ? 2 : 1)) + 3 * (b == 0 ? 0 : (b == ny - 1 ? 2 : 1));
            const std::complex<double>* v = G.v[cls];
            for (int db = -1; db <= 1; ++db)
                for (int da = -1; da <= 1; ++da) {
                    int la = a + da, lb = b + db;
                    if (la < 0 || la >= nx || lb < 0 || lb >= ny) continue;
                    std::complex<double> acc = v[(da + 1) + 3 * (db + 1)];
                    std::complex<double> ml = m_grid[la + (size_t)nx * lb];
                    if (ml != 0.0) {
                        std::complex<double> sum = 0;
                        for (int sb = -1; sb <= 1; ++sb)
                            for (int sa = -1; sa <= 1; ++sa) {
                                if (a + sa < 0 || a + sa >= nx || b + sb < 0 || b + sb >= ny) continue;
                                sum += v[(sa + 1) + 3 * (sb + 1)] * vcoff[(a + sa - la) + 2][(b + sb - lb) + 2];
                            }
                        acc += k2 * ml * sum;
                    }
                    G.cband[((size_t)b * 9 + (db + 1) * 3 + (da + 1)) * nx + a] = acc;
                }
        }
    return "";
}

}  // namespace lsgpu
