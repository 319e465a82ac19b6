// lattice.cuh -- compile-time lattice tables for the CUDA kernels.
//
// D3Q19: velocity set of eq. (HeLuoD3Q19), weights of eq. (omega) and the d'Humieres moment
// matrix T printed in Sec. 2 of the paper (rows in the order of the moment vector eq. (moment)).
// D2Q9: the Lallemand-Luo basis (the paper names D2Q9 but prints no table): velocities
// rest, +x, +y, -x, -y, (1,1), (-1,1), (-1,-1), (1,-1); rows 1, e = -4 + 3c^2,
// eps = 4 - 21c^2/2 + 9c^4/2, j_x, q_x = (-5 + 3c^2) c_x, j_y, q_y, p_xx = c_x^2 - c_y^2, p_xy.
// D3Q15: the d'Humieres et al. (2002) basis (the paper names D3Q15 but prints no table):
// velocities rest, +-x, +-y, +-z, then the corners (+-1, +-1, +-1) with c_x alternating fastest;
// rows 1, e = c^2 - 2, eps = (15c^4 - 55c^2 + 32)/2, j_x, q_x = (5c^2 - 13) c_x / 2, j_y, q_y, j_z,
// q_z, 3p_xx = 3c_x^2 - c^2, p_ww = c_y^2 - c_z^2, p_xy, p_yz, p_xz, m_xyz = c_x c_y c_z.
//
// Weights are wnum(i) / WDEN.
//
// Every table is a constexpr function so that fully unrolled loops fold each entry into the
// instruction stream (no constant-bank or local-memory lookups).
#pragma once

namespace lbm {

struct D3Q19 {
    static constexpr int Q = 19, D = 3, NS = 6, NP = 9;

    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr int C[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                  {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, 1, 0},  {1, -1, 0},
                                  {-1, -1, 0}, {1, 0, 1}, {-1, 0, 1}, {1, 0, -1},  {-1, 0, -1},
                                  {0, 1, 1},  {0, -1, 1}, {0, 1, -1}, {0, -1, -1}};
        return C[i][a];
    }
    __host__ __device__ static constexpr int T(int k, int i) {
        constexpr int M[19][19] = {
            {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
            {-30, -11, -11, -11, -11, -11, -11, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8},
            {12, -4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
            {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
            {0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
            {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
            {0, 0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
            {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
            {0, 0, 0, 0, 0, -4, 4, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
            {0, 2, 2, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
            {0, -4, -4, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
            {0, 0, 0, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
            {0, 0, 0, -2, -2, 2, 2, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
            {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 0, 0, 0, 0},
            {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1},
            {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0},
            {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1, 0, 0, 0, 0},
            {0, 0, 0, 0, 0, 0, 0, -1, -1, 1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
            {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1}};
        return M[k][i];
    }
    // weights: 1/3 rest, 1/18 axis, 1/36 edge
    static constexpr int WDEN = 36;
    __host__ __device__ static constexpr int wnum(int i) { return i == 0 ? 12 : (i <= 6 ? 2 : 1); }
    // opposite-velocity pairs (a, b) with c_b = -c_a
    __host__ __device__ static constexpr int pa(int p) {
        constexpr int A[9] = {1, 3, 5, 7, 8, 11, 12, 15, 16};
        return A[p];
    }
    __host__ __device__ static constexpr int pb(int p) {
        constexpr int B[9] = {2, 4, 6, 10, 9, 14, 13, 18, 17};
        return B[p];
    }
    __host__ __device__ static constexpr bool conserved(int k) { return k == 0 || k == 3 || k == 5 || k == 7; }
    __host__ __device__ static constexpr bool viscous(int k) {
        return k == 9 || k == 11 || k == 13 || k == 14 || k == 15;
    }
    static constexpr int NU0 = 9;  // first viscous moment
};

struct D2Q9 {
    static constexpr int Q = 9, D = 2, NS = 3, NP = 4;

    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr int C[9][3] = {{0, 0, 0}, {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
        return C[i][a];
    }
    __host__ __device__ static constexpr int T(int k, int i) {
        constexpr int M[9][9] = {{1, 1, 1, 1, 1, 1, 1, 1, 1},   {-4, -1, -1, -1, -1, 2, 2, 2, 2},
                                 {4, -2, -2, -2, -2, 1, 1, 1, 1}, {0, 1, 0, -1, 0, 1, -1, -1, 1},
                                 {0, -2, 0, 2, 0, 1, -1, -1, 1},  {0, 0, 1, 0, -1, 1, 1, -1, -1},
                                 {0, 0, -2, 0, 2, 1, 1, -1, -1},  {0, 1, -1, 1, -1, 0, 0, 0, 0},
                                 {0, 0, 0, 0, 0, 1, -1, 1, -1}};
        return M[k][i];
    }
    // weights 4/9, 1/9, 1/36
    static constexpr int WDEN = 36;
    __host__ __device__ static constexpr int wnum(int i) { return i == 0 ? 16 : (i <= 4 ? 4 : 1); }
    __host__ __device__ static constexpr int pa(int p) {
        constexpr int A[4] = {1, 2, 5, 6};
        return A[p];
    }
    __host__ __device__ static constexpr int pb(int p) {
        constexpr int B[4] = {3, 4, 7, 8};
        return B[p];
    }
    __host__ __device__ static constexpr bool conserved(int k) { return k == 0 || k == 3 || k == 5; }
    __host__ __device__ static constexpr bool viscous(int k) { return k == 7 || k == 8; }
    static constexpr int NU0 = 7;
};

struct D3Q15 {
    static constexpr int Q = 15, D = 3, NS = 6, NP = 7;

    __host__ __device__ static constexpr int c(int i, int a) {
        constexpr int C[15][3] = {{0, 0, 0},   {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                  {0, 0, 1},   {0, 0, -1}, {1, 1, 1},  {-1, 1, 1},  {1, -1, 1},
                                  {-1, -1, 1}, {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};
        return C[i][a];
    }
    __host__ __device__ static constexpr int T(int k, int i) {
        constexpr int M[15][15] = {{1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
                                   {-2, -1, -1, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1},
                                   {16, -4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1},
                                   {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1},
                                   {0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1},
                                   {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
                                   {0, 0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
                                   {0, 0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1},
                                   {0, 0, 0, 0, 0, -4, 4, 1, 1, 1, 1, -1, -1, -1, -1},
                                   {0, 2, 2, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
                                   {0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
                                   {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1},
                                   {0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1},
                                   {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1},
                                   {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, -1, 1, 1, -1}};
        return M[k][i];
    }
    // weights 2/9 rest, 1/9 axis, 1/72 corner
    static constexpr int WDEN = 72;
    __host__ __device__ static constexpr int wnum(int i) { return i == 0 ? 16 : (i <= 6 ? 8 : 1); }
    __host__ __device__ static constexpr int pa(int p) {
        constexpr int A[7] = {1, 3, 5, 7, 8, 9, 10};
        return A[p];
    }
    __host__ __device__ static constexpr int pb(int p) {
        constexpr int B[7] = {2, 4, 6, 14, 13, 12, 11};
        return B[p];
    }
    __host__ __device__ static constexpr bool conserved(int k) { return k == 0 || k == 3 || k == 5 || k == 7; }
    __host__ __device__ static constexpr bool viscous(int k) { return k >= 9 && k <= 13; }
    static constexpr int NU0 = 9;
};

// sum_i T_ki^2 (rows are orthogonal, so T^-1 = T^T diag(1/norm))
template <class L>
__host__ __device__ constexpr int norm2(int k) {
    int s = 0;
    for (int i = 0; i < L::Q; ++i) s += L::T(k, i) * L::T(k, i);
    return s;
}

// moment k is even (T_k,a == T_k,b on every opposite pair) or odd (T_k,a == -T_k,b)
template <class L>
__host__ __device__ constexpr bool even_moment(int k) {
    for (int p = 0; p < L::NP; ++p)
        if (L::T(k, L::pa(p)) != L::T(k, L::pb(p))) return false;
    return true;
}

template <class L>
__host__ __device__ constexpr bool odd_moment(int k) {
    if (L::T(k, 0) != 0) return false;
    for (int p = 0; p < L::NP; ++p)
        if (L::T(k, L::pa(p)) != -L::T(k, L::pb(p))) return false;
    return true;
}

template <class L>
__host__ __device__ constexpr bool basis_is_parity_split() {
    for (int k = 0; k < L::Q; ++k)
        if (!even_moment<L>(k) && !odd_moment<L>(k)) return false;
    for (int p = 0; p < L::NP; ++p)
        for (int a = 0; a < 3; ++a)
            if (L::c(L::pa(p), a) != -L::c(L::pb(p), a)) return false;
    return true;
}

static_assert(basis_is_parity_split<D3Q19>(), "D3Q19 basis must split into even and odd moments");
static_assert(basis_is_parity_split<D2Q9>(), "D2Q9 basis must split into even and odd moments");
static_assert(basis_is_parity_split<D3Q15>(), "D3Q15 basis must split into even and odd moments");

// the rows of T are orthogonal (T^-1 = T^T diag(1/norm2) is used by every back-transform)
template <class L>
__host__ __device__ constexpr bool rows_orthogonal() {
    for (int k = 0; k < L::Q; ++k)
        for (int l = k + 1; l < L::Q; ++l) {
            int s = 0;
            for (int i = 0; i < L::Q; ++i) s += L::T(k, i) * L::T(l, i);
            if (s != 0) return false;
        }
    return true;
}
static_assert(rows_orthogonal<D3Q19>() && rows_orthogonal<D2Q9>() && rows_orthogonal<D3Q15>(), "orthogonal bases");

}  // namespace lbm
