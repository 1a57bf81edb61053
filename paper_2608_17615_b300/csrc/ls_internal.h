// Internal data structures shared by the host setup (setup.cpp) and the
// device code (lsgpu.cu).  Not part of the public ABI.
#pragma once
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace lsgpu {

constexpr int NQ_ELEM = 15;   // nodes per element (interpolation degree p = 4)

struct HostMesh {
    int nv = 0, nt = 0, nq = 0, ncurve = 0;
    std::vector<double> vxy;      // [nv][2]
    std::vector<int> tri;         // [nt][3]
    std::vector<int> dom;         // [nt]
    std::vector<int> ecurve;      // [nt][3]
    std::vector<double> etheta;   // [nt][3][2]
    std::vector<double> curves;   // [ncurve][6]
    std::vector<double> nodes;    // [nq][2]
    std::vector<double> w;        // [nq]
};

struct CsrC {                     // complex CSR, int64 row pointers
    std::vector<int64_t> rowptr;
    std::vector<int32_t> cols;
    std::vector<std::complex<double>> vals;
};

// VDIM correction dV (local-patch form of Eq. DIM_decomp), extended precision.
// Returns "" on success, else an error message.
std::string build_correction(const HostMesh& mesh, double k, double kappa, CsrC& out);

// Work list of the device build of dV: one block per (target, subdomain with a patch),
// the blocks of a target consecutive and in the order of the host build's columns.
struct CorrPlan {
    std::vector<int64_t> row_blocks;           // [nq + 1] first block of each target
    std::vector<int32_t> target, tau;          // [nb] target node, interpolation element
    std::vector<int8_t> own;                   // [nb] target's own subdomain (chi = 1)
    std::vector<int64_t> elem_off;             // [nb + 1] into elems
    std::vector<int32_t> elems;                // patch elements
    std::vector<int64_t> pan_off;              // [nb + 1] into the panel arrays
    std::vector<int32_t> pan_edge;             // 3 element + local edge
    std::vector<long double> pan_a, pan_b;     // parameter interval of the panel on its edge
};
std::string plan_correction(const HostMesh& mesh, double kappa, CorrPlan& plan);
// Monomial centre/scale (cx, cy, 1/h) and coefficient matrices C, Phi [15 monomials][15 nodes]
// of the Lagrange basis of element tau and of its Helmholtz particular solutions.
bool poly_context(const HostMesh& mesh, int tau, double k, long double* c3, long double* C, long double* Phi);
// One block of dV by the host routine (extended precision): 15 values.
bool correction_block_host(const HostMesh& mesh, int j, double k, const std::vector<int>& patch, int tau, bool own,
                           std::complex<double>* out15);
// 32-point Gauss-Legendre rule on [0, 1] (long double).
void gl32_unit(long double* x, long double* w);
// The same dV built on the GPU (double-double moments, vdim_dev.cu); blocks whose patch
// leaves the series range are rebuilt on the host (their count in *host_blocks).
std::string build_correction_device(const HostMesh& mesh, double k, double kappa, void* stream, CsrC& out,
                                    int64_t* host_blocks);

struct GridSetup {
    int nx = 0, ny = 0;
    double x0 = 0, y0 = 0, h = 0;
    // T_C^Q: per quadrature node the 4 corner grid indices and bilinear weights
    std::vector<int32_t> tcq_idx;     // [nq][4]
    std::vector<double> tcq_w;        // [nq][4]
    // T_Q^C as a gather CSR over grid rows: Approach II weight psi_i(y_q) / D_i, or
    // Approach I the local L^2 projection (rows of interior grid nodes only)
    std::vector<int64_t> tqc_rowptr;  // [nx*ny + 1]
    std::vector<int32_t> tqc_cols;
    std::vector<double> tqc_vals;
    std::vector<double> D;            // [nx*ny]
    // (T_C^Q)^T as a gather CSR over grid rows (weights psi_i(y_q)), for P^T
    std::vector<int64_t> tcqT_rowptr;
    std::vector<int32_t> tcqT_cols;
    std::vector<double> tcqT_vals;
    // (T_Q^C)^T as a gather CSR over quadrature rows, for P^T
    std::vector<int64_t> tqcT_rowptr;  // [nq + 1]
    std::vector<int32_t> tqcT_cols;
    std::vector<double> tqcT_vals;
    int n_interior = 0;               // grid nodes inside an element (Approach I rows)
    // sparsifying stencils v[c][(da+1) + 3 (db+1)] per grid-row class c = ca + 3 cb
    // (0 / 1 / 2 = first / inner / last column or row); zero at offsets outside the grid
    std::complex<double> v[9][9];
    // C in block-tridiagonal form: [ny][3 (db)][3 (da)][nx]; entry C(j=(a,b), l=(a+da,b+db))
    std::vector<std::complex<double>> cband;
};

// Grid transfers, stencil and the banded C (Section 4).  "" on success.
std::string build_grid(const HostMesh& mesh, double k, const double box[4], int nx, int ny,
                       const std::complex<double>* m_grid, GridSetup& out, int approach = 2);
// The sparsifying stencils and the banded C on a grid with the given contrast (no mesh).
std::string build_stencil_C(double k, const double box[4], int nx, int ny, const std::complex<double>* m_grid,
                            GridSetup& out);
// V^(C) entries for offsets (a, b), 0 <= a < nx, 0 <= b < ny: K[b nx + a] (long double Hankel).
void cartesian_kernel_table(double k, double h, int nx, int ny, std::vector<std::complex<double>>& K);
// The transfer operators alone (T_C^Q, D, T_Q^C of the approach and the transposed CSRs).
std::string build_transfers(const HostMesh& mesh, const double box[4], int nx, int ny, int approach, GridSetup& out);

// Per-operator table of H0^(1)(k sqrt(t)) over t = r^2 for the pair sum.
// Octave [2^(B-1023), 2^(B-1022)) (B = biased exponent of t) is split into
// 2^m equal cells (m = 20 - shift); on each cell H0 is a degree-(NCOEF-1)
// polynomial in u = (t - mid) * inv_hw in [-1, 1] (monomial coefficients).
constexpr int H0TAB_NCOEF = 12;     // FP64 table: degree 11
struct H0Table {
    int b_lo = 0;                          // biased exponent of the first octave
    int noct = 0;
    std::vector<int> oct_base, oct_shift;  // [noct]
    std::vector<double> mid, inv_hw;       // [ncell]
    std::vector<std::complex<double>> coef;  // [ncell][H0TAB_NCOEF]
    double max_rel_err = 0;                // validated against the long-double routine
};
std::string build_h0_table(double k, double t_lo, double t_hi, H0Table& T, int ncoef = H0TAB_NCOEF,
                           double tol = 2e-15);

// Long-double Hankel functions used by the setup (host only).
void hankel01_ld(long double z, std::complex<long double>& h0, std::complex<long double>& h1);

}  // namespace lsgpu
