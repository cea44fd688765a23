// Pade-type high-order transmission operator of one interface side (host code, for
// the setup of an HABC transmission; Sections 3 and 6: HABCs as the transmission
// conditions, N_pade = 8 auxiliary fields, rotation phi = pi/3).
//
// The one-way operator d_n u = i k sqrt(1 + Lap_G / k^2) u with the square root by
// the rotated-branch Pade approximation of the HABC references,
//     sqrt(1 + z) ~ e^{i phi/2} R_N((1 + z) e^{-i phi} - 1),
//     R_N(w) = 1 + sum_l a_l w / (1 + b_l w),  a_l = 2/M sin^2(l pi/M),
//     b_l = cos^2(l pi/M),  M = 2N + 1
// (R_N the [N/N] Pade approximant of sqrt(1 + w) at 0; the rotation moves its branch
// cut so that evanescent modes are damped).  On the L points of a side, with Lap_G the
// 3-point second difference of spacing h and homogeneous Neumann ends and k the
// wavenumber of each point, the operator is the dense matrix
//     T = i diag(k) e^{i phi/2} R_N(W),  W = (I + diag(1/k^2) Lap_G) e^{-i phi} - I,
//     R_N(W) = I + sum_l a_l (I + b_l W)^{-1} W.
#include "helm_internal.cuh"

#include <cmath>
#include <complex>
#include <string>
#include <vector>

namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

// X <- A^{-1} X (A: n x n, X: n x m, both row-major; A is overwritten) by Gaussian
// elimination with partial pivoting; false when a pivot vanishes
bool solve_in_place(std::vector<cd>& A, std::vector<cd>& X, int n, int m) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::abs(A[(size_t)r * n + c]) > std::abs(A[(size_t)piv * n + c])) piv = r;
        if (std::abs(A[(size_t)piv * n + c]) == 0.0) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
            for (int k = 0; k < m; ++k) std::swap(X[(size_t)c * m + k], X[(size_t)piv * m + k]);
        }
        const cd inv = 1.0 / A[(size_t)c * n + c];
        for (int r = c + 1; r < n; ++r) {
            const cd f = A[(size_t)r * n + c] * inv;
            if (f == 0.0) continue;
            for (int k = c; k < n; ++k) A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
            for (int k = 0; k < m; ++k) X[(size_t)r * m + k] -= f * X[(size_t)c * m + k];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        const cd inv = 1.0 / A[(size_t)c * n + c];
        for (int k = 0; k < m; ++k) {
            cd v = X[(size_t)c * m + k];
            for (int j = c + 1; j < n; ++j) v -= A[(size_t)c * n + j] * X[(size_t)j * m + k];
            X[(size_t)c * m + k] = v * inv;
        }
    }
    return true;
}

}  // namespace

extern "C" helm_status helm_habc_side_operator(const double* kappa, int L, double h, int n_pade, double phi,
                                               helm_c128* T) {
    if (!kappa || !T || L < 1 || !(h > 0.0) || n_pade < 0) {
        set_error("helm_habc_side_operator: kappa and T non-NULL, L >= 1, h > 0 and n_pade >= 0 are required");
        return HELM_ERR_ARG;
    }
    for (int r = 0; r < L; ++r)
        if (!(kappa[r] > 0.0) || !std::isfinite(kappa[r])) {
            set_error("helm_habc_side_operator: every kappa must be positive and finite");
            return HELM_ERR_ARG;
        }
    const size_t LL = (size_t)L * L;
    const cd rot = std::polar(1.0, -phi);
    // W = (I + diag(1/k^2) Lap_G) e^{-i phi} - I
    std::vector<cd> W(LL, cd(0.0));
    for (int r = 0; r < L; ++r) {
        const double s = 1.0 / (kappa[r] * kappa[r] * h * h);
        const int ends = (r == 0) + (r == L - 1);          // Neumann: the ghost equals the end value
        W[(size_t)r * L + r] = (1.0 + s * (-2.0 + ends)) * rot - 1.0;
        if (r > 0) W[(size_t)r * L + r - 1] = s * rot;
        if (r < L - 1) W[(size_t)r * L + r + 1] = s * rot;
    }
    // R = I + sum_l a_l (I + b_l W)^{-1} W
    std::vector<cd> R(LL, cd(0.0));
    for (int r = 0; r < L; ++r) R[(size_t)r * L + r] = 1.0;
    const int M = 2 * n_pade + 1;
    for (int l = 1; l <= n_pade; ++l) {
        const double th = l * kPi / M;
        const double al = 2.0 / M * std::sin(th) * std::sin(th), bl = std::cos(th) * std::cos(th);
        std::vector<cd> A(LL), Y(W);
        for (size_t e = 0; e < LL; ++e) A[e] = bl * W[e];
        for (int r = 0; r < L; ++r) A[(size_t)r * L + r] += 1.0;
        if (!solve_in_place(A, Y, L, L)) {
            set_error("helm_habc_side_operator: singular factor I + b_l W");
            return HELM_ERR_ARG;
        }
        for (size_t e = 0; e < LL; ++e) R[e] += al * Y[e];
    }
    // T = i diag(k) e^{i phi/2} R
    const cd pre = cd(0.0, 1.0) * std::polar(1.0, 0.5 * phi);
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < L; ++c) {
            const cd v = pre * kappa[r] * R[(size_t)r * L + c];
            T[(size_t)r * L + c] = helm_c128{v.real(), v.imag()};
        }
    return HELM_OK;
}
