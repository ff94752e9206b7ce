// Host-side element data: the hex8 element matrix and its sum/difference form.
//
// The element stiffness (Sec. III: K_e = int_{Omega_e} k_e) of a trilinear
// hexahedron on the unit cube with isotropic material (E = 1, Poisson nu) is
// integrated exactly from the Lame bilinear form
//   a(u, v) = int lam div u div v + mu (grad u : grad v + grad u : grad v^T),
// which is separable: every entry is a product of three 1-D integrals of the
// hats 1 - t, t and their derivatives.
//
// In the basis of sums and differences of the element's 2x2x2 nodes
// (u^ = T u with T the tensor product of [1 1; -1 1]) the matrix
// K^ = T^-T K_e T^-1 = (1/64) T K_e T^T has 45 non-zeros; the operator kernels
// apply K_e as T^T (E_e K^) T, i.e. 3 x 24 butterfly adds, 45 products and
// 3 x 24 butterfly adds instead of a dense 24 x 24 product.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "internal.cuh"

namespace to {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

const char* last_error() { return g_last_error.c_str(); }

// Positions of the 45 non-zeros (row, col), grouped in the blocks that
// symmetry makes them fall into.
const int kHaarRow[kHaarNnz] = {
    3, 3, 3, 7, 7, 7, 14, 14, 14,       // normal strains  {ssd.x, sds.y, dss.z}
    4, 4, 6, 6,                         // shear xy        {ssd.y, sds.x}
    5, 5, 12, 12,                       // shear xz        {ssd.z, dss.x}
    8, 8, 13, 13,                       // shear yz        {sds.z, dss.y}
    9, 9, 20, 20,                       // {sdd.x, dds.z}
    10, 10, 17, 17,                     // {sdd.y, dsd.z}
    15, 15, 19, 19,                     // {dsd.x, dds.y}
    11, 11, 11, 16, 16, 16, 18, 18, 18, // {sdd.z, dsd.y, dds.x}
    21, 22, 23};                        // ddd
const int kHaarCol[kHaarNnz] = {
    3, 7, 14, 3, 7, 14, 3, 7, 14,
    4, 6, 4, 6,
    5, 12, 5, 12,
    8, 13, 8, 13,
    9, 20, 9, 20,
    10, 17, 10, 17,
    15, 19, 15, 19,
    11, 16, 18, 11, 16, 18, 11, 16, 18,
    21, 22, 23};

static const int kNodeOff[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                   {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};

// int_0^1 of (hat p or its derivative) * (hat q or its derivative)
static double hat_integral(int p, int q, bool dp, bool dq) {
    const double sp = p ? 1.0 : -1.0, sq = q ? 1.0 : -1.0;
    if (dp && dq) return sp * sq;
    if (dp) return 0.5 * sp;
    if (dq) return 0.5 * sq;
    return p == q ? 1.0 / 3.0 : 1.0 / 6.0;
}

// G_ij[a][b] = int d_i N_a d_j N_b over the unit cube
static double grad_product(int i, int j, int a, int b) {
    double v = 1.0;
    for (int d = 0; d < 3; ++d) v *= hat_integral(kNodeOff[a][d], kNodeOff[b][d], d == i, d == j);
    return v;
}

int build_element_matrix(double nu, double ke[24 * 24]) {
    if (!(nu >= 0.0 && nu < 0.5)) return fail(TO_ERR_ARG, "Poisson ratio must lie in [0, 0.5)");
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = 1.0 / (2.0 * (1.0 + nu));
    for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double v = lam * grad_product(i, j, a, b) + mu * grad_product(j, i, a, b);
                    if (i == j)
                        for (int k = 0; k < 3; ++k) v += mu * grad_product(k, k, a, b);
                    ke[(3 * a + i) * 24 + 3 * b + j] = v;
                }
    return TO_OK;
}

int build_haar(const double ke[24 * 24], double h, double out[kHaarNnz]) {
    // T[idx][l] = prod over axes of (sum: 1, difference: -1 at offset 0, +1 at offset 1)
    double T[8][8];
    for (int idx = 0; idx < 8; ++idx) {
        const int bit[3] = {idx & 1, (idx >> 1) & 1, (idx >> 2) & 1};  // x, y, z
        for (int l = 0; l < 8; ++l) {
            double v = 1.0;
            for (int d = 0; d < 3; ++d)
                if (bit[d]) v *= kNodeOff[l][d] ? 1.0 : -1.0;
            T[idx][l] = v;
        }
    }
    static double Kh[24][24];
    static std::mutex mtx;
    std::lock_guard<std::mutex> lock(mtx);
    double maxabs = 0.0;
    for (int r = 0; r < 24; ++r)
        for (int c = 0; c < 24; ++c) {
            const int ir = r / 3, cr = r % 3, ic = c / 3, cc = c % 3;
            double s = 0.0;
            for (int l = 0; l < 8; ++l)
                for (int m = 0; m < 8; ++m) s += T[ir][l] * ke[(3 * l + cr) * 24 + 3 * m + cc] * T[ic][m];
            Kh[r][c] = s / 64.0;
            maxabs = std::fmax(maxabs, std::fabs(Kh[r][c]));
        }
    bool used[24][24] = {};
    for (int n = 0; n < kHaarNnz; ++n) {
        used[kHaarRow[n]][kHaarCol[n]] = true;
        out[n] = h * Kh[kHaarRow[n]][kHaarCol[n]];
    }
    for (int r = 0; r < 24; ++r)
        for (int c = 0; c < 24; ++c)
            if (!used[r][c] && std::fabs(Kh[r][c]) > 1e-13 * maxabs) {
                char buf[160];
                std::snprintf(buf, sizeof buf, "element matrix has an unexpected non-zero (%d, %d) = %g in the sum/difference basis",
                              r, c, Kh[r][c]);
                return fail(TO_ERR_ARG, buf);
            }
    return TO_OK;
}

}  // namespace to

extern "C" const char* to_last_error(void) { return to::last_error(); }
