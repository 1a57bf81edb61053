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

struct GridSetup {
    int nx = 0, ny = 0;
    double x0 = 0, y0 = 0, h = 0;
    // T_C^Q: per quadrature node the 4 corner grid indices and bilinear weights
    std::vector<int32_t> tcq_idx;     // [nq][4]
    std::vector<double> tcq_w;        // [nq][4]
    // T_Q^C (Approach II) as a gather CSR over grid rows: weight psi_i(y_q) / D_i
    std::vector<int64_t> tqc_rowptr;  // [nx*ny + 1]
    std::vector<int32_t> tqc_cols;
    std::vector<double> tqc_vals;
    std::vector<double> D;            // [nx*ny]
    // sparsifying stencil v (3x3, index (da+1) + 3 (db+1))
    std::complex<double> v[9];
    // C in block-tridiagonal form: [ny][3 (db)][3 (da)][nx]; entry C(j=(a,b), l=(a+da,b+db))
    std::vector<std::complex<double>> cband;
};

// Grid transfers, stencil and the banded C (Section 4).  "" on success.
std::string build_grid(const HostMesh& mesh, double k, const double box[4], int nx, int ny,
                       const std::complex<double>* m_grid, GridSetup& out);

// Long-double Hankel functions used by the setup (host only).
void hankel01_ld(long double z, std::complex<long double>& h0, std::complex<long double>& h1);

}  // namespace lsgpu
