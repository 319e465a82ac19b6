// step.cuh -- the fused MRT lattice Boltzmann step and its read-out, init and sum kernels.
//
// A step pulls each node's 19 (or 9) pre-collision populations from the previous post-collision
// buffer (f_i(x) = f*_i(x - c_i), Sec. 2 eq. (mrteq)), forms S by Yu's formula (eq. (LuoS)) or
// Chai's formula (eq. (ChaiS)), solves the strain-rate closure for tau, relaxes in moment space
// (eq. (mrteqvT)) with the discrete force, and stores f* at the node: a single pass over HBM,
// 2 q values per node.
//
// Both routes write the collision in "delta form", f* = f - (increment), so that the
// storage-precision rounding acts only on the small collision increment:
//   Yu route:   D_k = (s_k mneq_k - TF_k) / |T_k|^2 over moments k, mneq = T f - m_eq + TF/2,
//               f*_i = f_i - sum_k T_ki D_k.
//   Chai route: fneq_i = f_i - f_eq_i + Fbar_i/2;  Omega = T^-1 L T fneq;
//               S = -sum_i c_i c_i Omega_i / (2 rho0 cs^2);  f*_i = f_i - Omega_i + Fbar_i.
// TF = T Fbar is the moment vector of the Guo-type discrete force Fbar_i =
// w_i[(c_i - u).F/cs^2 + (c_i.u)(c_i.F)/cs^4]; it equals the j-derivative of m_eq along F.
// With a closure the viscous rates are unknown, so both routes split S = A + s_nu B (exact:
// S is linear in the rates) and solve the scalar fixed point for tau = 1/s_nu.
//
// A thread owns one node (this file), or with 16-bit storage two x-adjacent nodes that share the
// pull's address arithmetic and collide side by side in packed FP32-pair arithmetic
// (step_pair.cuh, which forms f* from the post-collision moments instead of in delta form).
//
// All lattice coefficients enter as compile-time constants: loops over populations and moments
// are compile-time sequences (sfor) so each entry of T and c folds into an add, a subtract or
// an FMA with an immediate.  Accumulators start at -0.0, the exact additive identity, so the
// first term needs no special case.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "lattice.cuh"


namespace lbm {

enum { CL_NEWTON = 0, CL_SMAG = 1, CL_POWERLAW = 2, CL_SMAG_LAGGED = 3, CL_SMAG_DEV = 4 };
enum { F_YU = 0, F_CHAI = 1 };

// ------------------------------------------------------------------------------------------
// compile-time loops

template <class F, int... Is>
__host__ __device__ __forceinline__ void sfor_impl(F&& f, std::integer_sequence<int, Is...>) {
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__host__ __device__ __forceinline__ void sfor(F&& f) {
    sfor_impl(f, std::make_integer_sequence<int, N>{});
}
#define CV(x) (decltype(x)::value)

// fused multiply-add under one name for both compute types
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }

// the pulled populations of two x-adjacent nodes (lo: the even node, hi: the odd one)
struct F2 {
    float2 v;
    F2() = default;
    __device__ __forceinline__ F2(float a, float b) : v{a, b} {}
    __device__ __forceinline__ explicit F2(float2 u) : v(u) {}
    __device__ __forceinline__ float lo() const { return v.x; }
    __device__ __forceinline__ float hi() const { return v.y; }
};

// acc + t x for a compile-time integer t
template <int T, class R>
__device__ __forceinline__ R cadd(R acc, R x) {
    if constexpr (T == 0)
        return acc;
    else if constexpr (T == 1)
        return acc + x;
    else if constexpr (T == -1)
        return acc - x;
    else
        return fma(R(float(T)), x, acc);
}
template <class R>
__device__ __forceinline__ constexpr R nzero() {
    return R(-0.0f);
}
// a constant given in double, rounded once to the compute type (exact for the FP64 path)
template <class R>
__device__ __forceinline__ constexpr R cst(double c) {
    if constexpr (std::is_same<R, double>::value)
        return c;
    else
        return R(float(c));
}

// ------------------------------------------------------------------------------------------
// storage types: scalar access, and the pair load of the two-node path.  ld/ld2 read through
// the non-coherent path (the buffer is read-only for the whole kernel); ldc/ld2c read through L2
// only (ld.global.cg), for a kernel that reads populations other blocks of the same kernel wrote
// after synchronising with them.

template <class ST>
struct Store;
template <>
struct Store<double> {
    using R = double;
    static __device__ __forceinline__ R ld(const double* p) { return __ldg(p); }
    static __device__ __forceinline__ R ldc(const double* p) { return __ldcg(p); }
    static __device__ __forceinline__ void st(double* p, R v) { __stcs(p, v); }
};
template <>
struct Store<float> {
    using R = float;
    static __device__ __forceinline__ R ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ R ldc(const float* p) { return __ldcg(p); }
    static __device__ __forceinline__ void st(float* p, R v) { __stcs(p, v); }
    // aligned pair p[0], p[1] (p 8-byte aligned)
    static __device__ __forceinline__ F2 ld2(const float* p) { return F2(__ldg(reinterpret_cast<const float2*>(p))); }
    static __device__ __forceinline__ F2 ld2c(const float* p) { return F2(__ldcg(reinterpret_cast<const float2*>(p))); }
};
template <>
struct Store<__half> {
    using R = float;
    static __device__ __forceinline__ R ld(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ R ldc(const __half* p) { return __half2float(__ldcg(p)); }
    static __device__ __forceinline__ void st(__half* p, R v) { *p = __float2half_rn(v); }
    // aligned pair p[0] = lo, p[1] = hi (p 4-byte aligned), each rounded to nearest as st does
    static __device__ __forceinline__ void st2(__half* p, R lo, R hi) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(lo, hi);
    }
    static __device__ __forceinline__ F2 ld2(const __half* p) {
        return F2(__half22float2(__ldg(reinterpret_cast<const __half2*>(p))));
    }
    static __device__ __forceinline__ F2 ld2c(const __half* p) {
        return F2(__half22float2(__ldcg(reinterpret_cast<const __half2*>(p))));
    }
};
template <>
struct Store<__nv_bfloat16> {
    using R = float;
    static __device__ __forceinline__ R ld(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ R ldc(const __nv_bfloat16* p) { return __bfloat162float(__ldcg(p)); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, R v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ void st2(__nv_bfloat16* p, R lo, R hi) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(lo, hi);
    }
    static __device__ __forceinline__ F2 ld2(const __nv_bfloat16* p) {
        return F2(__bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p))));
    }
    static __device__ __forceinline__ F2 ld2c(const __nv_bfloat16* p) {
        return F2(__bfloat1622float2(__ldcg(reinterpret_cast<const __nv_bfloat162*>(p))));
    }
};

__device__ __forceinline__ float r_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double r_abs(double x) { return fabs(x); }
// Closure arithmetic: in FP32 the fast reciprocal / reciprocal-square-root / power intrinsics
// (errors of a few ulp, far inside the FP32 tolerance of S); in FP64 the IEEE operations.
__device__ __forceinline__ float c_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double c_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float c_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
__device__ __forceinline__ double c_sqrt(double x) { return sqrt(x); }
// |S|^(n-1) of the power-law closure from q2 = 2 S:S = |S|^2: in FP32 one fast power of q2 with
// exponent (n-1)/2 (no square root; exactly 1 for n = 1; a q2 rounded below zero counts as zero,
// as the square root's guard does), in FP64 the IEEE square root and power.
__device__ __forceinline__ float strain_pow(float q2, float nm1) {
    return nm1 == 0.0f ? 1.0f : __powf(fmaxf(q2, 0.0f), 0.5f * nm1);
}
__device__ __forceinline__ double strain_pow(double q2, double nm1) { return pow(sqrt(q2), nm1); }

// ------------------------------------------------------------------------------------------
// kernel arguments (by value; scalar type RS = float or double)

template <class RS>
struct StepArgs {
    int nx, ny, nz;
    int z0, nzc;           // planes computed: [z0, z0 + nzc) (all, or the owned planes between halo planes)
    int readout;           // 0: step (write f*); 1: write S/tau/drho/u of the pre-collision state
    long long stride;      // elements between population arrays
    const void* src;       // post-collision buffer of the previous step
    void* dst;             // post-collision buffer of this step
    const void* srcp[19];  // src + i * stride, population i (filled on the host)
    void* dstp[19];        // dst + i * stride
    const RS* force_field; // d x N, or nullptr for the uniform force F
    RS F[3];
    RS s[19];              // relaxation rates; the viscous entries hold 1/tau0
    RS skn[19];            // s_k / |T_k|^2
    RS rho0, inv_rho0, tau0;
    RS smag_c3;            // 3 Cs^2
    RS pl_k3, pl_nm1, pl_tau_min, pl_tau_max, pl_tol;  // 3K, n-1, clamp, tolerance
    int smag_iters, pl_max_iter;
    int wall_mask;         // bit f: face f is not periodic (wall or lid)
    int lid_mask;          // bit f: face f is a moving wall
    RS lid[6][3];
    RS* S_out;
    RS* tau_out;
    RS* drho_out;
    RS* u_out;
    RS* tau_field;         // lagged closure: N stored taus, read and rewritten in place by each node
};

// ------------------------------------------------------------------------------------------
// lattice-derived compile-time facts

template <class L>
__host__ __device__ constexpr int opp(int i) {
    for (int p = 0; p < L::NP; ++p) {
        if (L::pa(p) == i) return L::pb(p);
        if (L::pb(p) == i) return L::pa(p);
    }
    return i;
}

// strain components: xx, yy, zz, xy, yz, xz (3D) or xx, yy, xy (2D)
template <class L>
__host__ __device__ constexpr int strain_axis(int cpt, int which) {
    constexpr int ab3[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {1, 2}, {0, 2}};
    constexpr int ab2[3][2] = {{0, 0}, {1, 1}, {0, 1}};
    return L::NS == 6 ? ab3[cpt][which] : ab2[cpt][which];
}

// ------------------------------------------------------------------------------------------
// moment transforms

// m_K = sum_i T_Ki f_i from the rest population and the opposite-pair sums P / differences Dd
template <class L, int K, class R>
__device__ __forceinline__ R moment(R f0, const R (&P)[L::NP], const R (&Dd)[L::NP]) {
    R acc = nzero<R>();
    if constexpr (even_moment<L>(K)) {
        acc = cadd<L::T(K, 0)>(acc, f0);
        sfor<L::NP>([&](auto p) { acc = cadd<L::T(K, L::pa(CV(p)))>(acc, P[p]); });
    } else {
        sfor<L::NP>([&](auto p) { acc = cadd<L::T(K, L::pa(CV(p)))>(acc, Dd[p]); });
    }
    return acc;
}

// out_i = sum_k T_ki D_k over the moments k whose bit is set in USE, via even and odd parts of
// each opposite pair
template <class L, uint32_t USE, class R>
__device__ __forceinline__ void back_transform(const R (&D)[L::Q], R (&out)[L::Q]) {
    R r = nzero<R>();
    sfor<L::Q>([&](auto k) {
        if constexpr ((USE >> CV(k)) & 1u) r = cadd<L::T(CV(k), 0)>(r, D[k]);
    });
    out[0] = r;
    sfor<L::NP>([&](auto p) {
        constexpr int a = L::pa(CV(p)), b = L::pb(CV(p));
        R E = nzero<R>(), O = nzero<R>();
        sfor<L::Q>([&](auto k) {
            if constexpr ((USE >> CV(k)) & 1u) {
                if constexpr (even_moment<L>(CV(k)))
                    E = cadd<L::T(CV(k), a)>(E, D[k]);
                else
                    O = cadd<L::T(CV(k), a)>(O, D[k]);
            }
        });
        out[a] = E + O;
        out[b] = E - O;
    });
}

// Even and odd parts of out_i = sum_k T_ki D_k over the moments whose bit is set in USE: the rest
// population gets E0, and each opposite pair p = (a, b) gets out_a = E_p + O_p, out_b = E_p - O_p.
template <class L, uint32_t USE, class R>
__device__ __forceinline__ void back_transform_eo(const R (&D)[L::Q], R& E0, R (&E)[L::NP], R (&O)[L::NP]) {
    R r = nzero<R>();
    sfor<L::Q>([&](auto k) {
        if constexpr ((USE >> CV(k)) & 1u) r = cadd<L::T(CV(k), 0)>(r, D[k]);
    });
    E0 = r;
    sfor<L::NP>([&](auto p) {
        constexpr int a = L::pa(CV(p));
        R e = nzero<R>(), o = nzero<R>();
        sfor<L::Q>([&](auto k) {
            if constexpr ((USE >> CV(k)) & 1u) {
                if constexpr (even_moment<L>(CV(k)))
                    e = cadd<L::T(CV(k), a)>(e, D[k]);
                else
                    o = cadd<L::T(CV(k), a)>(o, D[k]);
            }
        });
        E[p] = e;
        O[p] = o;
    });
}

template <class L>
__host__ __device__ constexpr uint32_t mask_nonconserved() {
    uint32_t m = 0;
    for (int k = 0; k < L::Q; ++k)
        if (!L::conserved(k)) m |= 1u << k;
    return m;
}
template <class L>
__host__ __device__ constexpr uint32_t mask_viscous() {
    uint32_t m = 0;
    for (int k = 0; k < L::Q; ++k)
        if (L::viscous(k)) m |= 1u << k;
    return m;
}
template <class L>
__host__ __device__ constexpr uint32_t mask_all_but_density() {
    return ((1u << L::Q) - 1u) & ~1u;
}
template <class L>
__host__ __device__ constexpr uint32_t mask_all() {
    return (1u << L::Q) - 1u;
}

// Forward and backward transforms.  The generic form (any lattice) sums the nonzero entries of
// each row of T over the opposite-pair sums and differences.  D3Q19 and D3Q15 have hand-factored forms
// that share partial sums (axis / edge / corner butterflies) between rows; they compute the same maps.
template <class L>
struct Xf {
    // m[k] = (T f)_k for every k (m[0] = drho, m[3], m[5], m[7] = raw momentum)
    template <class R>
    static __device__ __forceinline__ void forward(R f0, const R (&P)[L::NP], const R (&Dd)[L::NP], R (&m)[L::Q]) {
        sfor<L::Q>([&](auto k) { m[k] = moment<L, CV(k)>(f0, P, Dd); });
    }
    template <uint32_t USE, class R>
    static __device__ __forceinline__ void backward(const R (&D)[L::Q], R (&out)[L::Q]) {
        back_transform<L, USE>(D, out);
    }
    template <uint32_t USE, class R>
    static __device__ __forceinline__ void backward_eo(const R (&D)[L::Q], R& E0, R (&E)[L::NP], R (&O)[L::NP]) {
        back_transform_eo<L, USE>(D, E0, E, O);
    }
};

template <>
struct Xf<D3Q19> {
    // pair order: x (1,2), y (3,4), z (5,6), (7,10), (8,9), (11,14), (12,13), (15,18), (16,17)

    // Even and odd parts of out_i = sum_k T_ki a_k (as back_transform_eo) for the two masks of the
    // Chai route, sharing partial sums between pairs: the non-conserved non-viscous moments
    // (1, 2, 4, 6, 8, 10, 12, 16, 17, 18) and the viscous moments (9, 11, 13, 14, 15, all even).
    // Other masks use the generic form.
    template <uint32_t USE, class R>
    static __device__ __forceinline__ void backward_eo(const R (&a)[19], R& E0, R (&E)[9], R (&O)[9]) {
        constexpr uint32_t FIXED = mask_nonconserved<D3Q19>() & ~mask_viscous<D3Q19>();
        constexpr uint32_t VISC = mask_viscous<D3Q19>();
        if constexpr (USE == FIXED) {
            E0 = fma(R(12.0f), a[2], R(-30.0f) * a[1]);
            const R B1 = fma(R(-4.0f), a[2], R(-11.0f) * a[1]);  // axis pairs
            const R B2 = fma(R(8.0f), a[1], a[2]);               // edge pairs
            const R s = a[10] + a[12], t = a[10] - a[12];
            E[0] = fma(R(-4.0f), a[10], B1);
            E[1] = fma(R(2.0f), t, B1);
            E[2] = fma(R(2.0f), s, B1);
            E[3] = E[4] = B2 + s;                                // xy edges
            E[5] = E[6] = B2 + t;                                // xz edges
            E[7] = E[8] = fma(R(-2.0f), a[10], B2);             // yz edges
            O[0] = R(-4.0f) * a[4];
            O[1] = R(-4.0f) * a[6];
            O[2] = R(-4.0f) * a[8];
            const R u1 = a[4] + a[16], v1 = a[6] - a[17];        // (7,10), (8,9)
            O[3] = v1 + u1;
            O[4] = v1 - u1;
            const R u2 = a[4] - a[16], v2 = a[8] + a[18];        // (11,14), (12,13)
            O[5] = v2 + u2;
            O[6] = v2 - u2;
            const R u3 = a[6] + a[17], v3 = a[8] - a[18];        // (15,18), (16,17)
            O[7] = v3 + u3;
            O[8] = v3 - u3;
        } else if constexpr (USE == VISC) {
            E0 = R(0.0f);
            const R p = a[9] + a[11], m = a[9] - a[11], t = R(-2.0f) * a[9];
            E[0] = R(2.0f) * a[9];
            E[1] = -m;
            E[2] = -p;
            E[3] = p + a[13];
            E[4] = p - a[13];
            E[5] = m + a[15];
            E[6] = m - a[15];
            E[7] = t + a[14];
            E[8] = t - a[14];
            sfor<9>([&](auto q) { O[q] = R(0.0f); });
        } else {
            back_transform_eo<D3Q19, USE>(a, E0, E, O);
        }
    }

    template <class R>
    static __device__ __forceinline__ void forward(R f0, const R (&P)[9], const R (&D)[9], R (&m)[19]) {
        const R Exy = P[3] + P[4], Exz = P[5] + P[6], Eyz = P[7] + P[8];
        const R Pyz = P[1] + P[2];
        const R Sax = P[0] + Pyz;
        const R Q = Exy + Exz;
        const R Sed = Q + Eyz;
        m[0] = f0 + Sax + Sed;
        const R Ex = (D[3] - D[4]) + (D[5] - D[6]);
        const R Ey = (D[3] + D[4]) + (D[7] - D[8]);
        const R Ez = (D[5] + D[6]) + (D[7] + D[8]);
        m[3] = D[0] + Ex;
        m[5] = D[1] + Ey;
        m[7] = D[2] + Ez;
        m[4] = fma(R(-4.0f), D[0], Ex);
        m[6] = fma(R(-4.0f), D[1], Ey);
        m[8] = fma(R(-4.0f), D[2], Ez);
        m[1] = fma(R(8.0f), Sed, fma(R(-11.0f), Sax, R(-30.0f) * f0));
        m[2] = fma(R(-4.0f), Sax, fma(R(12.0f), f0, Sed));
        const R Qm = fma(R(-2.0f), Eyz, Q);
        m[9] = fma(R(2.0f), P[0], Qm - Pyz);
        m[10] = fma(R(-4.0f), P[0], fma(R(2.0f), Pyz, Qm));
        const R dyz = P[1] - P[2], dxyz = Exy - Exz;
        m[11] = dyz + dxyz;
        m[12] = fma(R(-2.0f), dyz, dxyz);
        m[13] = P[3] - P[4];
        m[14] = P[7] - P[8];
        m[15] = P[5] - P[6];
        m[16] = (D[3] - D[4]) - (D[5] - D[6]);
        m[17] = (D[7] - D[8]) - (D[3] + D[4]);
        m[18] = (D[5] + D[6]) - (D[7] + D[8]);
    }

    // out_i = sum_k T_ki a_k.  The factored form needs every non-conserved a_k; with CONS the
    // momentum entries a_3, a_5, a_7 are included too (a_0 is always absent).  Other masks use
    // the generic form.
    template <uint32_t USE, class R>
    static __device__ __forceinline__ void backward(const R (&a)[19], R (&out)[19]) {
        constexpr uint32_t NC = mask_nonconserved<D3Q19>();
        if constexpr (USE != NC && USE != mask_all_but_density<D3Q19>() && USE != mask_all<D3Q19>()) {
            back_transform<D3Q19, USE>(a, out);
        } else {
            constexpr bool CONS = (USE >> 3) & 1u, DENS = USE & 1u;  // T_0i = 1 for every i
            out[0] = DENS ? fma(R(12.0f), a[2], fma(R(-30.0f), a[1], a[0])) : fma(R(12.0f), a[2], R(-30.0f) * a[1]);
            // axis populations
            const R B1 = DENS ? fma(R(-4.0f), a[2], fma(R(-11.0f), a[1], a[0])) : fma(R(-4.0f), a[2], R(-11.0f) * a[1]);
            const R C = fma(R(2.0f), a[10], -a[9]);
            const R W = fma(R(-2.0f), a[12], a[11]);
            const R Ex = fma(R(-2.0f), C, B1);
            const R BC = B1 + C;
            const R Ey = BC + W;
            const R Ez = BC - W;
            R Ox, Oy, Oz;
            if constexpr (CONS) {
                Ox = fma(R(-4.0f), a[4], a[3]);
                Oy = fma(R(-4.0f), a[6], a[5]);
                Oz = fma(R(-4.0f), a[8], a[7]);
            } else {
                Ox = R(-4.0f) * a[4];
                Oy = R(-4.0f) * a[6];
                Oz = R(-4.0f) * a[8];
            }
            out[1] = Ex + Ox;
            out[2] = Ex - Ox;
            out[3] = Ey + Oy;
            out[4] = Ey - Oy;
            out[5] = Ez + Oz;
            out[6] = Ez - Oz;
            // edge populations
            const R B2 = DENS ? fma(R(8.0f), a[1], a[2] + a[0]) : fma(R(8.0f), a[1], a[2]);
            const R G = a[9] + a[10], H = a[11] + a[12];
            R X = a[4], Y = a[6], Z = a[8];
            if constexpr (CONS) {
                X += a[3];
                Y += a[5];
                Z += a[7];
            }
            const R BG = B2 + G;
            {  // xy edges: (7,10) and (8,9)
                const R base = BG + H;
                const R E4 = base + a[13], E5 = base - a[13];
                const R u = X + a[16], v = Y - a[17];
                const R O4 = v + u, O5 = v - u;
                out[7] = E4 + O4;
                out[10] = E4 - O4;
                out[8] = E5 + O5;
                out[9] = E5 - O5;
            }
            {  // xz edges: (11,14) and (12,13)
                const R base = BG - H;
                const R E6 = base + a[15], E7 = base - a[15];
                const R u = X - a[16], v = Z + a[18];
                const R O6 = v + u, O7 = v - u;
                out[11] = E6 + O6;
                out[14] = E6 - O6;
                out[12] = E7 + O7;
                out[13] = E7 - O7;
            }
            {  // yz edges: (15,18) and (16,17)
                const R base = fma(R(-2.0f), G, B2);
                const R E8 = base + a[14], E9 = base - a[14];
                const R u = Y + a[17], v = Z - a[18];
                const R O8 = v + u, O9 = v - u;
                out[15] = E8 + O8;
                out[18] = E8 - O8;
                out[16] = E9 + O9;
                out[17] = E9 - O9;
            }
        }
    }
};

template <>
struct Xf<D3Q15> {
    // pair order: x (1,2), y (3,4), z (5,6), corners (7,14), (8,13), (9,12), (10,11); the four corner
    // pairs are combined by two-level butterflies shared between rows
    template <class R>
    static __device__ __forceinline__ void forward(R f0, const R (&P)[7], const R (&D)[7], R (&m)[15]) {
        const R a = P[3] + P[6], b = P[4] + P[5], c = P[3] - P[6], d = P[4] - P[5];
        const R Sc = a + b, Sax = P[0] + (P[1] + P[2]);
        const R u = D[3] + D[5], v = D[4] + D[6], w = D[3] - D[5], x = D[4] - D[6];
        const R Cx = u - v, Cy = w + x, Cz = u + v;
        m[0] = f0 + Sax + Sc;
        m[1] = fma(R(-2.0f), f0, Sc - Sax);
        m[2] = fma(R(16.0f), f0, fma(R(-4.0f), Sax, Sc));
        m[3] = D[0] + Cx;
        m[4] = fma(R(-4.0f), D[0], Cx);
        m[5] = D[1] + Cy;
        m[6] = fma(R(-4.0f), D[1], Cy);
        m[7] = D[2] + Cz;
        m[8] = fma(R(-4.0f), D[2], Cz);
        m[9] = fma(R(3.0f), P[0], -Sax);
        m[10] = P[1] - P[2];
        m[11] = a - b;
        m[12] = c + d;
        m[13] = c - d;
        m[14] = w - x;
    }

    // Even and odd parts of out_i = sum_k T_ki a_k for the Chai route's two masks: the
    // non-conserved non-viscous moments (1, 2, 4, 6, 8, 14) and the viscous moments (9..13, all
    // even), with the corner pairs as butterflies; other masks use the generic form.
    template <uint32_t USE, class R>
    static __device__ __forceinline__ void backward_eo(const R (&a)[15], R& E0, R (&E)[7], R (&O)[7]) {
        constexpr uint32_t FIXED = mask_nonconserved<D3Q15>() & ~mask_viscous<D3Q15>();
        constexpr uint32_t VISC = mask_viscous<D3Q15>();
        if constexpr (USE == FIXED) {
            E0 = fma(R(16.0f), a[2], R(-2.0f) * a[1]);
            E[0] = E[1] = E[2] = fma(R(-4.0f), a[2], -a[1]);   // axis pairs
            E[3] = E[4] = E[5] = E[6] = a[1] + a[2];           // corner pairs
            O[0] = R(-4.0f) * a[4];
            O[1] = R(-4.0f) * a[6];
            O[2] = R(-4.0f) * a[8];
            const R p = a[8] + a[6], m = a[8] - a[6], c = a[4] + a[14], d = a[4] - a[14];
            O[3] = p + c;  // (7,14): c = (1, 1, 1)
            O[4] = p - c;  // (8,13): (-1, 1, 1)
            O[5] = m + d;  // (9,12): (1, -1, 1)
            O[6] = m - d;  // (10,11): (-1, -1, 1)
        } else if constexpr (USE == VISC) {
            E0 = R(0.0f);
            E[0] = R(2.0f) * a[9];
            E[1] = a[10] - a[9];
            E[2] = -(a[9] + a[10]);
            const R s1 = a[11] + a[13], s2 = a[11] - a[13];
            E[3] = a[12] + s1;
            E[4] = a[12] - s1;
            E[5] = -(a[12] + s2);
            E[6] = s2 - a[12];
            sfor<7>([&](auto q) { O[q] = R(0.0f); });
        } else {
            back_transform_eo<D3Q15, USE>(a, E0, E, O);
        }
    }

    // out_i = sum_k T_ki a_k for every non-conserved a_k (with CONS also a_3, a_5, a_7); other
    // masks use the generic form
    template <uint32_t USE, class R>
    static __device__ __forceinline__ void backward(const R (&a)[15], R (&out)[15]) {
        constexpr uint32_t NC = mask_nonconserved<D3Q15>();
        if constexpr (USE != NC && USE != mask_all_but_density<D3Q15>() && USE != mask_all<D3Q15>()) {
            back_transform<D3Q15, USE>(a, out);
        } else {
            constexpr bool CONS = (USE >> 3) & 1u, DENS = USE & 1u;  // T_0i = 1 for every i
            out[0] = DENS ? fma(R(16.0f), a[2], fma(R(-2.0f), a[1], a[0])) : fma(R(16.0f), a[2], R(-2.0f) * a[1]);
            // axis populations
            const R B1 = DENS ? fma(R(-4.0f), a[2], a[0] - a[1]) : fma(R(-4.0f), a[2], -a[1]);
            const R Ex = fma(R(2.0f), a[9], B1), BC = B1 - a[9];
            const R Ey = BC + a[10], Ez = BC - a[10];
            R Ox, Oy, Oz, X = a[4], Y = a[6], Z = a[8];
            if constexpr (CONS) {
                Ox = fma(R(-4.0f), a[4], a[3]);
                Oy = fma(R(-4.0f), a[6], a[5]);
                Oz = fma(R(-4.0f), a[8], a[7]);
                X += a[3];
                Y += a[5];
                Z += a[7];
            } else {
                Ox = R(-4.0f) * a[4];
                Oy = R(-4.0f) * a[6];
                Oz = R(-4.0f) * a[8];
            }
            out[1] = Ex + Ox;
            out[2] = Ex - Ox;
            out[3] = Ey + Oy;
            out[4] = Ey - Oy;
            out[5] = Ez + Oz;
            out[6] = Ez - Oz;
            // corner populations: even parts B2 +- a11 +- a12 +- a13, odd parts +-X +-Y +-Z +- a14
            const R B2 = DENS ? (a[1] + a[2]) + a[0] : a[1] + a[2];
            const R s = B2 + a[11], t = B2 - a[11], g = a[12] + a[13], h = a[12] - a[13];
            const R U = Z + Y, V = Z - Y, p = X + a[14], r = a[14] - X;
            const R E3 = s + g, E6 = s - g, E4 = t + h, E5 = t - h;
            const R O3 = U + p, O4 = U - p, O5 = V - r, O6 = V + r;
            out[7] = E3 + O3;
            out[14] = E3 - O3;
            out[8] = E4 + O4;
            out[13] = E4 - O4;
            out[9] = E5 + O5;
            out[12] = E5 - O5;
            out[10] = E6 + O6;
            out[11] = E6 - O6;
        }
    }
};

// N_c = sum_i c_ia c_ib v_i for each strain component c = (a, b)
template <class L, class R>
__device__ __forceinline__ void contract(const R (&v)[L::Q], R (&N)[L::NS]) {
    sfor<L::NS>([&](auto cpt) {
        constexpr int a = strain_axis<L>(CV(cpt), 0), b = strain_axis<L>(CV(cpt), 1);
        R acc = nzero<R>();
        sfor<L::Q>([&](auto i) { acc = cadd<L::c(CV(i), a) * L::c(CV(i), b)>(acc, v[i]); });
        N[cpt] = acc;
    });
}

// N_c = sum_i c_ia c_ib v_i for a field given by its opposite-pair even parts E_p: c_ia c_ib is
// even under c -> -c, so the odd parts cancel and each pair counts twice (the rest has c = 0).
template <class L, class R>
__device__ __forceinline__ void contract_even(const R (&E)[L::NP], R (&N)[L::NS]) {
    sfor<L::NS>([&](auto cpt) {
        constexpr int a = strain_axis<L>(CV(cpt), 0), b = strain_axis<L>(CV(cpt), 1);
        R acc = nzero<R>();
        sfor<L::NP>([&](auto p) {
            acc = cadd<L::c(L::pa(CV(p)), a) * L::c(L::pa(CV(p)), b)>(acc, E[p]);
        });
        N[cpt] = R(2.0f) * acc;
    });
}

template <class L>
__host__ __device__ constexpr bool viscous_moments_even() {
    for (int k = 0; k < L::Q; ++k)
        if (L::viscous(k) && !even_moment<L>(k)) return false;
    return true;
}

// ------------------------------------------------------------------------------------------
// equilibrium moments (closed form) and force moments TF = d m_eq / d j . F, both written with
// u = j / rho0 formed once

template <class L>
struct Eq;

template <>
struct Eq<D3Q19> {
    // eq. (meq): w_eps = 3, w_epsj = -11/2, w_xx = -1/2
    template <class R>
    static __device__ __forceinline__ void meq(R drho, const R (&j)[3], const R (&u)[3], R (&m)[19]) {
        const R ju = fma(j[0], u[0], fma(j[1], u[1], j[2] * u[2]));
        m[0] = drho;
        m[1] = fma(R(19.0f), ju, R(-11.0f) * drho);
        m[2] = fma(R(-5.5f), ju, R(3.0f) * drho);
        m[3] = j[0];
        m[4] = cst<R>(-2.0 / 3.0) * j[0];
        m[5] = j[1];
        m[6] = cst<R>(-2.0 / 3.0) * j[1];
        m[7] = j[2];
        m[8] = cst<R>(-2.0 / 3.0) * j[2];
        m[9] = fma(R(3.0f) * j[0], u[0], -ju);
        m[10] = R(-0.5f) * m[9];
        m[11] = fma(j[1], u[1], -(j[2] * u[2]));
        m[12] = R(-0.5f) * m[11];
        m[13] = j[0] * u[1];
        m[14] = j[1] * u[2];
        m[15] = j[0] * u[2];
        m[16] = R(0.0f);
        m[17] = R(0.0f);
        m[18] = R(0.0f);
    }
    template <class R>
    static __device__ __forceinline__ void tforce(const R (&u)[3], const R (&F)[3], R (&t)[19]) {
        const R uF = fma(u[0], F[0], fma(u[1], F[1], u[2] * F[2]));
        t[0] = R(0.0f);
        t[1] = R(38.0f) * uF;
        t[2] = R(-11.0f) * uF;
        t[3] = F[0];
        t[4] = cst<R>(-2.0 / 3.0) * F[0];
        t[5] = F[1];
        t[6] = cst<R>(-2.0 / 3.0) * F[1];
        t[7] = F[2];
        t[8] = cst<R>(-2.0 / 3.0) * F[2];
        t[9] = fma(R(6.0f) * u[0], F[0], R(-2.0f) * uF);
        t[10] = R(-0.5f) * t[9];
        t[11] = R(2.0f) * fma(u[1], F[1], -(u[2] * F[2]));
        t[12] = R(-0.5f) * t[11];
        t[13] = fma(u[0], F[1], u[1] * F[0]);
        t[14] = fma(u[1], F[2], u[2] * F[1]);
        t[15] = fma(u[0], F[2], u[2] * F[0]);
        t[16] = R(0.0f);
        t[17] = R(0.0f);
        t[18] = R(0.0f);
    }
    // moments with identically zero equilibrium and force parts (ghost moments t_x, t_y, t_z)
    static __host__ __device__ constexpr bool ghost(int k) { return k >= 16; }
    // Yu formula eq. (LuoS) split as S = A + s_nu B (A: the s1 m1 part); c1 = s1/(38 rho0), ir0 = 1/rho0
    template <class R>
    static __device__ __forceinline__ void yu_split(const R (&mn)[19], R c1, R ir0, R (&A)[6], R (&B)[6]) {
        const R a = -(c1 * mn[1]);
        A[0] = a;
        A[1] = a;
        A[2] = a;
        A[3] = R(0.0f);
        A[4] = R(0.0f);
        A[5] = R(0.0f);
        const R h = R(0.25f) * ir0;
        const R k = R(-1.5f) * ir0;
        B[0] = (R(-0.5f) * ir0) * mn[9];
        B[1] = h * fma(R(-3.0f), mn[11], mn[9]);
        B[2] = h * fma(R(3.0f), mn[11], mn[9]);
        B[3] = k * mn[13];
        B[4] = k * mn[14];
        B[5] = k * mn[15];
    }
    static constexpr double YU_A = 1.0 / 38.0;  // c1 = s1 * YU_A / rho0
};

template <>
struct Eq<D3Q15> {
    // T f_eq of the He-Luo equilibrium on the d'Humieres D3Q15 basis
    template <class R>
    static __device__ __forceinline__ void meq(R drho, const R (&j)[3], const R (&u)[3], R (&m)[15]) {
        const R ju = fma(j[0], u[0], fma(j[1], u[1], j[2] * u[2]));
        m[0] = drho;
        m[1] = ju - drho;
        m[2] = fma(R(-5.0f), ju, drho);
        m[3] = j[0];
        m[4] = cst<R>(-7.0 / 3.0) * j[0];
        m[5] = j[1];
        m[6] = cst<R>(-7.0 / 3.0) * j[1];
        m[7] = j[2];
        m[8] = cst<R>(-7.0 / 3.0) * j[2];
        m[9] = fma(R(3.0f) * j[0], u[0], -ju);
        m[10] = fma(j[1], u[1], -(j[2] * u[2]));
        m[11] = j[0] * u[1];
        m[12] = j[1] * u[2];
        m[13] = j[0] * u[2];
        m[14] = R(0.0f);
    }
    template <class R>
    static __device__ __forceinline__ void tforce(const R (&u)[3], const R (&F)[3], R (&t)[15]) {
        const R uF = fma(u[0], F[0], fma(u[1], F[1], u[2] * F[2]));
        t[0] = R(0.0f);
        t[1] = R(2.0f) * uF;
        t[2] = R(-10.0f) * uF;
        t[3] = F[0];
        t[4] = cst<R>(-7.0 / 3.0) * F[0];
        t[5] = F[1];
        t[6] = cst<R>(-7.0 / 3.0) * F[1];
        t[7] = F[2];
        t[8] = cst<R>(-7.0 / 3.0) * F[2];
        t[9] = fma(R(6.0f) * u[0], F[0], R(-2.0f) * uF);
        t[10] = R(2.0f) * fma(u[1], F[1], -(u[2] * F[2]));
        t[11] = fma(u[0], F[1], u[1] * F[0]);
        t[12] = fma(u[1], F[2], u[2] * F[1]);
        t[13] = fma(u[0], F[2], u[2] * F[0]);
        t[14] = R(0.0f);
    }
    // m_xyz has zero equilibrium and force parts
    static __host__ __device__ constexpr bool ghost(int k) { return k == 14; }
    // Yu-type D3Q15 formula (Sec. 5.4 procedure): S_xx = -(s_e m_e + s_nu m_3pxx)/(2 rho0),
    // S_yy,zz = -(2 s_e m_e - s_nu m_3pxx +- 3 s_nu m_pww)/(4 rho0), S_ab = -3 s_nu m_pab/(2 rho0);
    // c1 = s_e/(2 rho0)
    template <class R>
    static __device__ __forceinline__ void yu_split(const R (&mn)[15], R c1, R ir0, R (&A)[6], R (&B)[6]) {
        const R a = -(c1 * mn[1]);
        A[0] = a;
        A[1] = a;
        A[2] = a;
        A[3] = R(0.0f);
        A[4] = R(0.0f);
        A[5] = R(0.0f);
        const R h = R(0.25f) * ir0;
        const R k = R(-1.5f) * ir0;
        B[0] = (R(-0.5f) * ir0) * mn[9];
        B[1] = h * fma(R(-3.0f), mn[10], mn[9]);
        B[2] = h * fma(R(3.0f), mn[10], mn[9]);
        B[3] = k * mn[11];
        B[4] = k * mn[12];
        B[5] = k * mn[13];
    }
    static constexpr double YU_A = 1.0 / 2.0;
};

template <>
struct Eq<D2Q9> {
    template <class R>
    static __device__ __forceinline__ void meq(R drho, const R (&j)[3], const R (&u)[3], R (&m)[9]) {
        const R ju = fma(j[0], u[0], j[1] * u[1]);
        m[0] = drho;
        m[1] = fma(R(3.0f), ju, R(-2.0f) * drho);
        m[2] = fma(R(-3.0f), ju, drho);
        m[3] = j[0];
        m[4] = -j[0];
        m[5] = j[1];
        m[6] = -j[1];
        m[7] = fma(j[0], u[0], -(j[1] * u[1]));
        m[8] = j[0] * u[1];
    }
    template <class R>
    static __device__ __forceinline__ void tforce(const R (&u)[3], const R (&F)[3], R (&t)[9]) {
        const R uF = fma(u[0], F[0], u[1] * F[1]);
        t[0] = R(0.0f);
        t[1] = R(6.0f) * uF;
        t[2] = R(-6.0f) * uF;
        t[3] = F[0];
        t[4] = -F[0];
        t[5] = F[1];
        t[6] = -F[1];
        t[7] = R(2.0f) * fma(u[0], F[0], -(u[1] * F[1]));
        t[8] = fma(u[0], F[1], u[1] * F[0]);
    }
    static __host__ __device__ constexpr bool ghost(int) { return false; }
    // Yu-type D2Q9 formula (Sec. 5.4 procedure): S_xx,yy = -(s_e m_e +- 3 s_nu m_pxx)/(4 rho0),
    // S_xy = -3 s_nu m_pxy / (2 rho0);  c1 = s_e/(4 rho0)
    template <class R>
    static __device__ __forceinline__ void yu_split(const R (&mn)[9], R c1, R ir0, R (&A)[3], R (&B)[3]) {
        const R a = -(c1 * mn[1]);
        A[0] = a;
        A[1] = a;
        A[2] = R(0.0f);
        const R h = R(0.75f) * ir0;
        B[0] = -(h * mn[7]);
        B[1] = h * mn[7];
        B[2] = (R(-1.5f) * ir0) * mn[8];
    }
    static constexpr double YU_A = 1.0 / 4.0;
};

// Chai route: the effective non-equilibrium distributions f - f_eq + Fbar/2 of the He-Luo
// equilibrium (eq. (edf)) and the Guo-type force, in opposite-pair form, formed directly.  With
// cj = c.j, cu = c.u, cF = c.F (c = c_a of pair p, weight w), g = u.(j - F) and
// B = 2 drho - 3 g, f_eq_a + f_eq_b = 2w (drho + 4.5 cj cu - 1.5 j.u), f_eq_a - f_eq_b = 6 w cj,
// Fbar_a + Fbar_b = 2w (9 cu cF - 3 u.F), Fbar_a - Fbar_b = 6 w cF, Fbar_0 = -3 w0 u.F, so that
//   (f_eq - Fbar/2)_a + (f_eq - Fbar/2)_b = w B + 9 w cu (cj - cF),
//   (f_eq - Fbar/2)_a - (f_eq - Fbar/2)_b = 3 w (2 cj - cF),
//   (f_eq - Fbar/2)_0 = w0 B / 2.
// Pn_p = P_p - (first), Dn_p = D_p - (second), fn0 = f0 - (third).
template <class L, bool FORCE, class R>
__device__ __forceinline__ void noneq_pairs(R f0, const R (&P)[L::NP], const R (&Dd)[L::NP], R drho, const R (&j)[3],
                                            const R (&u)[3], const R (&F)[3], R& fn0, R (&Pn)[L::NP],
                                            R (&Dn)[L::NP]) {
    R g = fma(j[0], u[0], fma(j[1], u[1], j[2] * u[2]));
    if constexpr (FORCE) g = fma(-u[0], F[0], fma(-u[1], F[1], fma(-u[2], F[2], g)));
    const R B = fma(R(-3.0f), g, R(2.0f) * drho);
    constexpr double w0 = double(L::wnum(0)) / L::WDEN;
    fn0 = fma(cst<R>(-0.5 * w0), B, f0);
    sfor<L::NP>([&](auto p) {
        constexpr int i = L::pa(CV(p));
        constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        constexpr double w = double(L::wnum(i)) / L::WDEN;
        const R cj = cadd<cz>(cadd<cy>(cadd<cx>(nzero<R>(), j[0]), j[1]), j[2]);
        const R cu = cadd<cz>(cadd<cy>(cadd<cx>(nzero<R>(), u[0]), u[1]), u[2]);
        R t = cj, t2 = R(2.0f) * cj;
        if constexpr (FORCE) {
            const R cF = cadd<cz>(cadd<cy>(cadd<cx>(nzero<R>(), F[0]), F[1]), F[2]);
            t = cj - cF;
            t2 = fma(R(2.0f), cj, -cF);
        }
        Pn[p] = fma(cst<R>(-9.0 * w) * cu, t, fma(cst<R>(-w), B, P[p]));
        Dn[p] = fma(cst<R>(-3.0 * w), t2, Dd[p]);
    });
}

// f <- f - Omega_f + Fbar for the Chai route, Omega_f given by its opposite-pair even / odd parts
// (Ef0 for the rest population), Fbar the Guo-type discrete force in the pair form above.
template <class L, bool FORCE, class R>
__device__ __forceinline__ void fold_fixed_part(R (&f)[L::Q], R Ef0, const R (&Ef)[L::NP], const R (&Of)[L::NP],
                                                const R (&u)[3], const R (&F)[3]) {
    constexpr double w0 = double(L::wnum(0)) / L::WDEN;
    R uF = R(0.0f);
    if constexpr (FORCE) {
        uF = fma(u[0], F[0], fma(u[1], F[1], u[2] * F[2]));
        f[0] = fma(cst<R>(-3.0 * w0), uF, f[0] - Ef0);
    } else {
        f[0] -= Ef0;
    }
    sfor<L::NP>([&](auto p) {
        constexpr int i = L::pa(CV(p));
        constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        constexpr double w = double(L::wnum(i)) / L::WDEN;
        R e = Ef[p], o = Of[p];
        if constexpr (FORCE) {
            const R cu = cadd<cz>(cadd<cy>(cadd<cx>(nzero<R>(), u[0]), u[1]), u[2]);
            const R cF = cadd<cz>(cadd<cy>(cadd<cx>(nzero<R>(), F[0]), F[1]), F[2]);
            e -= fma(cst<R>(9.0 * w) * cu, cF, cst<R>(-3.0 * w) * uF);  // Fbar even part / 2
            o = fma(cst<R>(-3.0 * w), cF, o);                            // Fbar odd part / 2
        }
        f[L::pa(CV(p))] -= e + o;
        f[L::pb(CV(p))] -= e - o;
    });
}

// The Guo-type discrete force Fbar_i (pair form above), population by population.
template <class L, class R>
__device__ __forceinline__ void force_bar(const R (&u)[3], const R (&F)[3], R (&Fb)[L::Q]) {
    constexpr double w0 = double(L::wnum(0)) / L::WDEN;
    const R uF = fma(u[0], F[0], fma(u[1], F[1], u[2] * F[2]));
    Fb[0] = cst<R>(-3.0 * w0) * uF;
    sfor<L::NP>([&](auto p) {
        constexpr int i = L::pa(CV(p));
        constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        constexpr double w = double(L::wnum(i)) / L::WDEN;
        const R cu = cadd<cz>(cadd<cy>(cadd<cx>(nzero<R>(), u[0]), u[1]), u[2]);
        const R cF = cadd<cz>(cadd<cy>(cadd<cx>(nzero<R>(), F[0]), F[1]), F[2]);
        const R e = fma(cst<R>(9.0 * w) * cu, cF, cst<R>(-3.0 * w) * uF), o = cst<R>(3.0 * w) * cF;
        Fb[L::pa(CV(p))] = e + o;
        Fb[L::pb(CV(p))] = e - o;
    });
}

// ------------------------------------------------------------------------------------------
// closure: solve tau with S = A + (1/tau) B

template <class L, class R>
__device__ __forceinline__ R strain_dot(const R (&S)[L::NS], const R (&T)[L::NS]) {
    // S:T with the off-diagonal components counted twice
    if constexpr (L::NS == 6)
        return fma(S[0], T[0], fma(S[1], T[1], S[2] * T[2])) +
               R(2.0f) * fma(S[3], T[3], fma(S[4], T[4], S[5] * T[5]));
    else
        return fma(S[0], T[0], S[1] * T[1]) + R(2.0f) * (S[2] * T[2]);
}

template <class L, class R>
__device__ __forceinline__ void affine(const R (&A)[L::NS], const R (&B)[L::NS], R s, R (&S)[L::NS]) {
#pragma unroll
    for (int c = 0; c < L::NS; ++c) S[c] = fma(s, B[c], A[c]);
}

// Fixed point for tau at one node from the quadratic |S|^2 = 2 (qa + qb2 s + qc s^2), s = 1/tau
// (qa = A:A, qb2 = 2 A:B, qc = B:B: exact since S = A + s B).  Smagorinsky: `smag_iters` sweeps
// from tau0, stopping early only when a sweep returns its input bit for bit (every later sweep
// would too).  Power law: sweeps until |tau_new - tau| <= pl_tol tau_new or pl_max_iter sweeps.
template <int CLOSURE, class RS>
__device__ __forceinline__ RS tau_fixed_point(RS qa, RS qb2, RS qc, const StepArgs<RS>& a) {
    RS tau = a.tau0;
    if constexpr (CLOSURE == CL_SMAG) {
        for (int it = 0; it < a.smag_iters; ++it) {
            const RS s = c_rcp(tau);
            const RS tn = fma(a.smag_c3, c_sqrt(RS(2) * fma(fma(qc, s, qb2), s, qa)), a.tau0);
            if (tn == tau) break;
            tau = tn;
        }
    } else {
        for (int it = 1; it <= a.pl_max_iter; ++it) {
            const RS s = c_rcp(tau);
            RS tn = fma(a.pl_k3, strain_pow(RS(2) * fma(fma(qc, s, qb2), s, qa), a.pl_nm1), RS(0.5));
            if (!(tn >= a.pl_tau_min)) tn = a.pl_tau_min;
            if (tn > a.pl_tau_max) tn = a.pl_tau_max;
            const RS diff = r_abs(tn - tau);
            tau = tn;
            if (diff <= a.pl_tol * tn) break;
        }
    }
    return tau;
}

// L2 eviction priority for per-node fields that every step reads again while the populations
// stream past: the force field (read-only) and the lagged closure's stored tau (read and rewritten
// by its own node each step).  Their loads and stores carry an evict_last policy, so the field
// (12 or 4 B per node in FP32) stays in L2 across the steps of a launch instead of coming from HBM
// every step.  A hint only: the data are the same either way.  Measured on a GB300: one 25 MB
// field stays (the same loads without the policy run at the old speed); two such fields hinted
// at once in the adjoint's reverse step (force field and gradient accumulator) both kept
// streaming from HBM, so only the force field carries the hint there.
__device__ __forceinline__ unsigned long long l2_keep() {
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// read-only field (non-coherent path), evict_last in L2
template <class RS>
__device__ __forceinline__ RS ld_keep(const RS* p) {
    const unsigned long long pol = l2_keep();
    if constexpr (std::is_same<RS, double>::value) {
        double v;
        asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
        return v;
    } else {
        float v;
        asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
        return v;
    }
}
// an aligned FP32 pair (p 8-byte aligned) of a read-only field, evict_last in L2
__device__ __forceinline__ float2 ld2_keep(const float* p) {
    const unsigned long long pol = l2_keep();
    float2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
// a field value written by another block earlier in the launch: loaded through L2 (asm volatile,
// so its issue point stays where it is written) and stored back, both evict_last in L2
template <class RS>
__device__ __forceinline__ RS load_early_keep(const RS* p) {
    const unsigned long long pol = l2_keep();
    if constexpr (std::is_same<RS, double>::value) {
        double v;
        asm volatile("ld.global.cg.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
        return v;
    } else {
        float v;
        asm volatile("ld.global.cg.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
        return v;
    }
}
// the same load without the eviction policy
template <class RS>
__device__ __forceinline__ RS load_early(const RS* p) {
    if constexpr (std::is_same<RS, double>::value) {
        double v;
        asm volatile("ld.global.cg.f64 %0, [%1];" : "=d"(v) : "l"(p));
        return v;
    } else {
        float v;
        asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(p));
        return v;
    }
}
template <class RS>
__device__ __forceinline__ void st_keep(RS* p, RS v) {
    const unsigned long long pol = l2_keep();
    if constexpr (std::is_same<RS, double>::value)
        asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
    else
        asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}

// Deviatoric Smagorinsky, tau = tau0 + 3 Cs^2 |S_d(1/tau)|.  On these bases the rate-free part A is
// isotropic and B is traceless, so S_d = s B and tau is the larger root of
// tau^2 - tau0 tau - 3 Cs^2 |B| = 0, |B| = sqrt(2 B:B).
template <class RS>
__device__ __forceinline__ RS tau_deviatoric(RS qc, const StepArgs<RS>& a) {
    const RS b = c_sqrt(RS(2) * qc);
    return RS(0.5) * (a.tau0 + c_sqrt(fma(a.tau0, a.tau0, RS(4) * a.smag_c3 * b)));
}

// Returns tau, sets snu = 1/tau and S = A + snu B.  The lagged closure collides with tau_prev, the
// tau stored at `node` (loaded by the caller together with the populations), and in a step (not a
// read-out) stores tau0 + 3 Cs^2 |S| there for the next step.
template <class L, class R, int CLOSURE, class RS>
__device__ __forceinline__ R solve_tau(const R (&A)[L::NS], const R (&B)[L::NS], const StepArgs<RS>& a,
                                       R (&S)[L::NS], R& snu, int node, R tau_prev = R(0.0f)) {
    if constexpr (CLOSURE == CL_NEWTON) {
        snu = R(a.s[L::NU0]);
        affine<L>(A, B, snu, S);
        return R(a.tau0);
    } else if constexpr (CLOSURE == CL_SMAG_LAGGED) {
        const R tau = tau_prev;
        snu = c_rcp(tau);
        affine<L>(A, B, snu, S);
        if (!a.readout) st_keep(a.tau_field + node, RS(fma(a.smag_c3, c_sqrt(RS(2) * strain_dot<L>(S, S)), a.tau0)));
        return tau;
    } else if constexpr (CLOSURE == CL_SMAG_DEV) {
        const R tau = tau_deviatoric(strain_dot<L>(B, B), a);
        snu = c_rcp(tau);
        affine<L>(A, B, snu, S);
        return tau;
    } else {
        const R qa = strain_dot<L>(A, A), qb2 = R(2.0f) * strain_dot<L>(A, B), qc = strain_dot<L>(B, B);
        const R tau = tau_fixed_point<CLOSURE>(qa, qb2, qc, a);
        snu = c_rcp(tau);
        affine<L>(A, B, snu, S);
        return tau;
    }
}

// ------------------------------------------------------------------------------------------
// pull streaming

// Pre-collision populations of node (x,y,z).  Interior rows (y, z away from the faces, and x
// away from non-periodic x faces) read population i at node + (x wrap) - c_iy nx - c_iz nx ny,
// the last two terms being the same for the whole warp; nodes on a periodic boundary row or plane
// with no wall next to them read the same way with the y and z wraps applied by index (a separate
// branch, so the interior code stays as short); the rest take the general rule:
// periodic faces wrap, a population whose source lies behind a wall is reflected from the
// opposite population of the same node, plus the moving-wall term when it crosses exactly one
// moving face.
template <class L, class ST, class RS>
__device__ __forceinline__ bool interior_rows(const StepArgs<RS>& a, int xlo, int xhi, int y, int z) {
    const bool xwall = (a.wall_mask & 3) != 0;
    bool fast = y > 0 && y < a.ny - 1 && (!xwall || (xlo > 0 && xhi < a.nx - 1));
    if constexpr (L::D == 3) fast = fast && z > 0 && z < a.nz - 1;
    return fast;
}

// no wall face next to the node (its periodic faces wrap by index)
template <class L, class ST, class RS>
__device__ __forceinline__ bool no_wall_next(const StepArgs<RS>& a, int x, int y, int z) {
    const int w = a.wall_mask;  // bit f: face f (-x, +x, -y, +y, -z, +z) is a wall
    bool ok = !(w & 3) || (x > 0 && x < a.nx - 1);
    ok = ok && (!(w & 12) || (y > 0 && y < a.ny - 1));
    if constexpr (L::D == 3) ok = ok && (!(w & 48) || (z > 0 && z < a.nz - 1));
    return ok;
}

// neighbour offsets along y and z with the periodic wrap: the source of c = +1 is one step back
struct WrapYZ {
    int ym, yp, zm, zp;
    __device__ __forceinline__ WrapYZ(int y, int z, int nx, int ny, int nz) {
        const int nxy = nx * ny;
        ym = y == 0 ? (ny - 1) * nx : -nx;
        yp = y == ny - 1 ? -(ny - 1) * nx : nx;
        zm = z == 0 ? (nz - 1) * nxy : -nxy;
        zp = z == nz - 1 ? -(nz - 1) * nxy : nxy;
    }
    template <int cy, int cz>
    __device__ __forceinline__ int off() const {
        return (cy > 0 ? ym : (cy < 0 ? yp : 0)) + (cz > 0 ? zm : (cz < 0 ? zp : 0));
    }
};

// population load: COH selects the coherent (L2) path
template <bool COH, class ST>
__device__ __forceinline__ typename Store<ST>::R ldp(const ST* p) {
    if constexpr (COH)
        return Store<ST>::ldc(p);
    else
        return Store<ST>::ld(p);
}
template <bool COH, class ST>
__device__ __forceinline__ F2 ldp2(const ST* p) {
    if constexpr (COH)
        return Store<ST>::ld2c(p);
    else
        return Store<ST>::ld2(p);
}

template <class L, class ST, bool COH = false, class RS>
__device__ __forceinline__ void pull_general(const StepArgs<RS>& a, int x, int y, int z, RS (&f)[L::Q],
                                             long long es = 0) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int node = (z * ny + y) * nx + x;
    const int dims[3] = {nx, ny, nz};
    const int pos[3] = {x, y, z};
    sfor<L::Q>([&](auto i) {
        int s[3];
        int nout = 0, face = -1;
        sfor<3>([&](auto ax) {
            constexpr int cax = L::c(CV(i), CV(ax));
            s[ax] = pos[ax] - cax;
            if constexpr (cax != 0) {
                if (s[ax] < 0 || s[ax] >= dims[ax]) {
                    const int fc = 2 * CV(ax) + (s[ax] < 0 ? 0 : 1);
                    if ((a.wall_mask >> fc) & 1) {
                        ++nout;
                        face = fc;
                    } else {
                        s[ax] = s[ax] < 0 ? s[ax] + dims[ax] : s[ax] - dims[ax];
                    }
                }
            }
        });
        if (nout == 0) {
            f[i] = ldp<COH>(static_cast<const ST*>(a.srcp[CV(i)]) + es + ((s[2] * ny + s[1]) * nx + s[0]));
        } else {
            RS v = ldp<COH>(static_cast<const ST*>(a.srcp[opp<L>(CV(i))]) + es + node);
            if (nout == 1 && ((a.lid_mask >> face) & 1)) {
                const RS cu = RS(L::c(CV(i), 0)) * a.lid[face][0] + RS(L::c(CV(i), 1)) * a.lid[face][1] +
                              RS(L::c(CV(i), 2)) * a.lid[face][2];
                v += RS(double(6 * L::wnum(CV(i))) / L::WDEN) * a.rho0 * cu;  // 2 w_i rho0 (c.u)/cs^2 = 6 w_i rho0 c.u
            }
            f[i] = v;
        }
    });
}

template <class L, class ST, bool COH = false, class RS>
__device__ __forceinline__ void pull(const StepArgs<RS>& a, int x, int y, int z, RS (&f)[L::Q], long long es = 0) {
    const int nx = a.nx, nxy = a.nx * a.ny;
    const int node = z * nxy + y * nx + x;
    const int dxm = x == 0 ? nx - 1 : -1;      // source of c_x = +1: x - 1 (wrapped)
    const int dxp = x == nx - 1 ? 1 - nx : 1;  // source of c_x = -1: x + 1 (wrapped)
    if (interior_rows<L, ST>(a, x, x, y, z)) {
        sfor<L::Q>([&](auto i) {
            constexpr int cx = L::c(CV(i), 0), cy = L::c(CV(i), 1), cz = L::c(CV(i), 2);
            const int off = node + (cx > 0 ? dxm : (cx < 0 ? dxp : 0)) - (cy * nx + cz * nxy);
            f[i] = ldp<COH>(static_cast<const ST*>(a.srcp[CV(i)]) + es + off);
        });
        return;
    }
    if (no_wall_next<L, ST>(a, x, y, z)) {  // on a periodic boundary row or plane: wrap y and z too
        const WrapYZ w(y, z, nx, a.ny, a.nz);
        sfor<L::Q>([&](auto i) {
            constexpr int cx = L::c(CV(i), 0), cy = L::c(CV(i), 1), cz = L::c(CV(i), 2);
            const int off = node + (cx > 0 ? dxm : (cx < 0 ? dxp : 0)) + w.template off<cy, cz>();
            f[i] = ldp<COH>(static_cast<const ST*>(a.srcp[CV(i)]) + es + off);
        });
        return;
    }
    pull_general<L, ST, COH>(a, x, y, z, f, es);
}

// Two nodes (x0, x0 + 1), x0 even, nx even: populations with c_x = 0 come as one aligned pair,
// the others as two scalar loads (x wrap applied per node); periodic boundary rows and planes
// with no wall next to either node wrap y and z by index, as in the one-node pull.
template <class L, class ST, bool COH = false>
__device__ __forceinline__ void pull2(const StepArgs<float>& a, int x0, int y, int z, F2 (&f)[L::Q]) {
    const int nx = a.nx, nxy = a.nx * a.ny;
    const int node = z * nxy + y * nx + x0;
    if (interior_rows<L, ST>(a, x0, x0 + 1, y, z)) {
        const int dxm = x0 == 0 ? nx - 1 : -1;          // node 0, c_x = +1: x0 - 1 (wrapped)
        const int dxp = x0 + 2 == nx ? 2 - nx : 2;      // node 1, c_x = -1: x0 + 2 (wrapped)
        sfor<L::Q>([&](auto i) {
            constexpr int cx = L::c(CV(i), 0), cy = L::c(CV(i), 1), cz = L::c(CV(i), 2);
            const ST* p = static_cast<const ST*>(a.srcp[CV(i)]) + (node - (cy * nx + cz * nxy));
            if constexpr (cx == 0)
                f[i] = ldp2<COH>(p);
            else if constexpr (cx > 0)
                f[i] = F2(ldp<COH>(p + dxm), ldp<COH>(p));
            else
                f[i] = F2(ldp<COH>(p + 1), ldp<COH>(p + dxp));
        });
        return;
    }
    if (no_wall_next<L, ST>(a, x0, y, z) && no_wall_next<L, ST>(a, x0 + 1, y, z)) {
        // on a periodic boundary row or plane: the same loads with the y and z wraps by index
        const WrapYZ w(y, z, nx, a.ny, a.nz);
        const int dxm = x0 == 0 ? nx - 1 : -1;
        const int dxp = x0 + 2 == nx ? 2 - nx : 2;
        sfor<L::Q>([&](auto i) {
            constexpr int cx = L::c(CV(i), 0), cy = L::c(CV(i), 1), cz = L::c(CV(i), 2);
            const ST* p = static_cast<const ST*>(a.srcp[CV(i)]) + (node + w.template off<cy, cz>());
            if constexpr (cx == 0)
                f[i] = ldp2<COH>(p);
            else if constexpr (cx > 0)
                f[i] = F2(ldp<COH>(p + dxm), ldp<COH>(p));
            else
                f[i] = F2(ldp<COH>(p + 1), ldp<COH>(p + dxp));
        });
        return;
    }
    float f0[L::Q], f1[L::Q];
    pull_general<L, ST, COH>(a, x0, y, z, f0);
    pull_general<L, ST, COH>(a, x0 + 1, y, z, f1);
    sfor<L::Q>([&](auto i) { f[i] = F2(f0[i], f1[i]); });
}

// ------------------------------------------------------------------------------------------
// the fused step

// Programmatic dependent launch.  A step launched with the programmatic-serialization attribute
// may become resident while the previous kernel of the stream is finishing; griddepcontrol.wait
// returns once that kernel has completed and its memory operations are visible, so it precedes
// every load.  launch_dependents lets the next such step be scheduled as soon as every block of
// this one has issued it; issued at block start, that happens once the last blocks are resident,
// so waiting blocks of the next step only take slots freed by this one.  Launched without the
// attribute, both instructions have no effect.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Everything of a step after the pull, for the node(s) starting at `node`: moments, strain rate
// by the chosen route, closure, relaxation, force, and either the store of f* or (readout) the
// store of S, tau, drho and u.  ds shifts the populations' destination by that many elements (a
// launch that writes each step to its own buffer of a ring); the pull's es does the same for the
// source.
template <class L, class ST, int CLOSURE, int FORMULA, bool FORCE>
__device__ __forceinline__ void step_body(const StepArgs<typename Store<ST>::R>& a, typename Store<ST>::R (&f)[L::Q],
                                          int node, long long ds = 0) {
    using RS = typename Store<ST>::R;
    using R = RS;
    constexpr int Q = L::Q, NS = L::NS, NP = L::NP;
    const long long N = (long long)a.nx * a.ny * a.nz;  // component offsets c*N exceed 2^31 on big grids

    R P[NP], Dd[NP];
    sfor<NP>([&](auto p) {
        P[p] = f[L::pa(CV(p))] + f[L::pb(CV(p))];
        Dd[p] = f[L::pa(CV(p))] - f[L::pb(CV(p))];
    });
    R F[3] = {R(0.0f), R(0.0f), R(0.0f)};
    if constexpr (FORCE) {
        if (a.force_field) {
            sfor<L::D>([&](auto d) { F[d] = ld_keep(a.force_field + CV(d) * N + node); });
        } else {
            sfor<L::D>([&](auto d) { F[d] = R(a.F[d]); });
        }
    }
    // the lagged closure's stored tau, loaded next to the populations so its latency overlaps theirs
    // (an asm volatile load keeps it there instead of next to its use after the moment arithmetic)
    R tau_prev = R(0.0f);
    if constexpr (CLOSURE == CL_SMAG_LAGGED) tau_prev = load_early_keep(a.tau_field + node);
    const R ir0 = R(a.inv_rho0);
    R drho, j[3] = {R(0.0f), R(0.0f), R(0.0f)}, u[3] = {R(0.0f), R(0.0f), R(0.0f)};
    R S[NS], tau, snu;
    R out[Q];  // f*_i = f_i - out_i

    if constexpr (FORMULA == F_YU) {
        // Yu route: moments of f, closed-form equilibrium moments, S from six of them
        R m[Q];
        Xf<L>::forward(f[0], P, Dd, m);
        drho = m[0];
        j[0] = FORCE ? fma(R(0.5f), F[0], m[3]) : m[3];
        j[1] = FORCE ? fma(R(0.5f), F[1], m[5]) : m[5];
        if constexpr (L::D == 3) j[2] = FORCE ? fma(R(0.5f), F[2], m[7]) : m[7];
        sfor<L::D>([&](auto d) { u[d] = j[d] * ir0; });
        // non-equilibrium moments; every collision increment D_k that does not involve the unknown
        // viscous rate is finished before the closure, so only the viscous moments (and their force
        // terms) stay live across the fixed point
        R Dk[Q], mn[Q], tv[Q];
        {
            R meq[Q], TF[Q];
            Eq<L>::meq(drho, j, u, meq);
            if constexpr (FORCE) Eq<L>::tforce(u, F, TF);
            sfor<Q>([&](auto k) {
                constexpr double inv_n = 1.0 / norm2<L>(CV(k));
                if constexpr (L::conserved(CV(k))) {
                    mn[k] = R(0.0f);
                    if constexpr (FORCE)
                        Dk[k] = cst<R>(-inv_n) * TF[k];
                    else
                        Dk[k] = R(0.0f);
                } else {
                    if constexpr (Eq<L>::ghost(CV(k)))
                        mn[k] = m[k];
                    else if constexpr (FORCE)
                        mn[k] = fma(R(0.5f), TF[k], m[k] - meq[k]);
                    else
                        mn[k] = m[k] - meq[k];
                    const bool has_tf = FORCE && !Eq<L>::ghost(CV(k));
                    if constexpr (L::viscous(CV(k))) {
                        tv[k] = has_tf ? cst<R>(-inv_n) * TF[k] : R(0.0f);
                    } else {
                        if constexpr (FORCE && !Eq<L>::ghost(CV(k)))
                            Dk[k] = fma(R(a.skn[k]), mn[k], cst<R>(-inv_n) * TF[k]);
                        else
                            Dk[k] = R(a.skn[k]) * mn[k];
                    }
                }
            });
        }
        R A[NS], B[NS];
        Eq<L>::yu_split(mn, R(a.s[1] * RS(Eq<L>::YU_A)) * ir0, ir0, A, B);
        tau = solve_tau<L, R, CLOSURE>(A, B, a, S, snu, node, tau_prev);
        if (a.readout) goto readout;
        sfor<Q>([&](auto k) {
            if constexpr (L::viscous(CV(k))) {
                constexpr double inv_n = 1.0 / norm2<L>(CV(k));
                if constexpr (FORCE)
                    Dk[k] = fma(snu * cst<R>(inv_n), mn[k], tv[k]);
                else
                    Dk[k] = (snu * cst<R>(inv_n)) * mn[k];
            }
        });
        // with a force, the conserved moments 3, 5, 7 (D2Q9: 3, 5) carry -TF_k; TF_0 = 0
        Xf<L>::template backward<FORCE ? mask_all_but_density<L>() : mask_nonconserved<L>()>(Dk, out);
    } else {
        // Chai route: non-equilibrium distributions f - f_eq + Fbar/2 (in opposite-pair form), the
        // collision operator T^-1 L T applied to them, and the second velocity moment of the result
        drho = f[0];
        sfor<NP>([&](auto p) { drho += P[p]; });
        sfor<L::D>([&](auto d) {
            R acc = nzero<R>();
            sfor<NP>([&](auto p) { acc = cadd<L::c(L::pa(CV(p)), CV(d))>(acc, Dd[p]); });
            j[d] = FORCE ? fma(R(0.5f), F[d], acc) : acc;
            u[d] = j[d] * ir0;
        });
        R fn0, Pn[NP], Dn[NP];
        noneq_pairs<L, FORCE>(f[0], P, Dd, drho, j, u, F, fn0, Pn, Dn);
        R mn[Q];
        Xf<L>::forward(fn0, Pn, Dn, mn);
        const R kS = R(-1.5f) * ir0;  // S = -N / (2 rho0 cs2)
        R Om[Q];                       // Omega (Newtonian) or its rate-independent part
        if constexpr (CLOSURE == CL_NEWTON) {
            R Dk[Q];
            sfor<Q>([&](auto k) {
                if constexpr (L::conserved(CV(k)))
                    Dk[k] = R(0.0f);
                else
                    Dk[k] = R(a.skn[k]) * mn[k];
            });
            Xf<L>::template backward<mask_nonconserved<L>()>(Dk, Om);
            R N[NS];
            contract<L>(Om, N);
#pragma unroll
            for (int c = 0; c < NS; ++c) S[c] = kS * N[c];
            tau = R(a.tau0);
            snu = R(a.s[L::NU0]);
            if (a.readout) goto readout;
            sfor<Q>([&](auto i) { out[i] = Om[i]; });
            if constexpr (FORCE) {  // f* = f - Omega + Fbar
                R Fb[Q];
                force_bar<L>(u, F, Fb);
                sfor<Q>([&](auto i) { out[i] -= Fb[i]; });
            }
        } else {
            R Df[Q], Dv[Q];
            sfor<Q>([&](auto k) {
                constexpr double inv_n = 1.0 / norm2<L>(CV(k));
                if constexpr (L::conserved(CV(k)) || L::viscous(CV(k)))
                    Df[k] = R(0.0f);
                else
                    Df[k] = R(a.skn[k]) * mn[k];
                if constexpr (L::viscous(CV(k)))
                    Dv[k] = cst<R>(inv_n) * mn[k];
                else
                    Dv[k] = R(0.0f);
            });
            // Omega = Omega_f + s_nu Omega_v in opposite-pair even / odd parts; the viscous moments
            // are all even, so Omega_v has no odd part, and S needs only the even parts
            static_assert(viscous_moments_even<L>(), "viscous moments must be even");
            R Ef0, Ef[NP], Of[NP], Ev0, Ev[NP], Ovd[NP];
            Xf<L>::template backward_eo<mask_nonconserved<L>() & ~mask_viscous<L>()>(Df, Ef0, Ef, Of);
            Xf<L>::template backward_eo<mask_viscous<L>()>(Dv, Ev0, Ev, Ovd);
            R Nf[NS], Nv[NS], A[NS], B[NS];
            contract_even<L>(Ef, Nf);
            contract_even<L>(Ev, Nv);
#pragma unroll
            for (int c = 0; c < NS; ++c) {
                A[c] = kS * Nf[c];
                B[c] = kS * Nv[c];
            }
            // f* = f - Omega_f + Fbar - s_nu Omega_v: everything but the last term is folded into f
            // now, so only f and Omega_v stay live across the closure
            fold_fixed_part<L, FORCE>(f, Ef0, Ef, Of, u, F);
            tau = solve_tau<L, R, CLOSURE>(A, B, a, S, snu, node, tau_prev);
            if (a.readout) goto readout;
            out[0] = snu * Ev0;
            sfor<NP>([&](auto p) {
                const R e = snu * Ev[p];
                out[L::pa(CV(p))] = e;
                out[L::pb(CV(p))] = e;
            });
        }
    }

    sfor<Q>([&](auto i) { Store<ST>::st(static_cast<ST*>(a.dstp[CV(i)]) + ds + node, f[i] - out[i]); });
    return;

readout:
    if (a.S_out) {
#pragma unroll
        for (int c = 0; c < NS; ++c) a.S_out[c * N + node] = S[c];
    }
    if (a.tau_out) a.tau_out[node] = tau;
    if (a.drho_out) a.drho_out[node] = drho;
    if (a.u_out) {
#pragma unroll
        for (int d = 0; d < L::D; ++d) a.u_out[d * N + node] = u[d];
    }
}

// One node per thread.  The bound names no minimum of resident blocks for the 3D lattices and
// FP64: a minimum of one changes ptxas's register allocation (more registers, fewer resident
// blocks).  FP32 D2Q9 is held to 16 blocks (32 registers, full occupancy), where the power-law
// closure otherwise took 40-45 registers: with the one-power closure above, +4% on a 4096^2
// power-law cavity (n = 0.5 and 1.5, both routes).
template <class L, class ST>
constexpr int step_min_blocks() {
    return (L::Q == 9 && sizeof(ST) == 4) ? 16 : 0;
}

template <class L, class ST, int CLOSURE, int FORMULA, bool FORCE>
__global__ void __launch_bounds__(128, step_min_blocks<L, ST>()) k_step(const StepArgs<typename Store<ST>::R> a) {
    pdl_wait();     // the previous step's stores are complete and visible from here on
    pdl_release();  // every block has started: the next step may be scheduled into freed slots
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z + a.z0;
    if (x >= a.nx || y >= a.ny) return;
    typename Store<ST>::R f[L::Q];
    pull<L, ST>(a, x, y, z, f);
    step_body<L, ST, CLOSURE, FORMULA, FORCE>(a, f, (z * a.ny + y) * a.nx + x);
}

// ------------------------------------------------------------------------------------------
// initialisation from (drho, u, grad u), computed in double, un-streamed into the buffer

template <class L, class ST>
__global__ void __launch_bounds__(128) k_init(const StepArgs<double> a, int closure, const double* __restrict__ drho,
                                              const double* __restrict__ u, const double* __restrict__ gu,
                                              const typename Store<ST>::R* __restrict__ ffield,
                                              typename Store<ST>::R* __restrict__ tau_field) {
    using R = typename Store<ST>::R;
    constexpr int Q = L::Q, D = L::D;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z + a.z0;
    if (x >= a.nx || y >= a.ny) return;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long N = (long long)nx * ny * nz;  // component offsets (up to 8N) exceed 2^31 on big grids
    const int node = (z * ny + y) * nx + x;
    const double r0 = a.rho0, ir0 = a.inv_rho0;
    double j[3] = {0, 0, 0}, F[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) j[d] = r0 * u[d * N + node];
    for (int d = 0; d < D; ++d) F[d] = ffield ? double(ffield[d * N + node]) : a.F[d];
    const double dr = drho[node];
    // first-order viscous non-equilibrium moments of the given gradient (D3Q19: eq. (YuLuobasis);
    // D2Q9 and D3Q15: the same first-order Chapman-Enskog moments worked out on their bases)
    double mn[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) mn[k] = 0.0;
    // the closure's tau at the prescribed gradient (explicit, since S is given); the lagged
    // closure stores it as the tau of the first step
    double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (gu)
        for (int p = 0; p < D; ++p)
            for (int q = 0; q < D; ++q) G[p][q] = r0 * gu[(p * D + q) * N + node];
    double tau_i = a.tau0;
    if (closure != CL_NEWTON) {
        double ss, tr = 0.0;
        if (closure == CL_SMAG_DEV) tr = (G[0][0] + G[1][1] + G[2][2]) / D;  // traceless part only
        const double e0 = G[0][0] - tr, e1 = G[1][1] - tr, e2 = D == 3 ? G[2][2] - tr : 0.0;
        if (D == 3)
            ss = e0 * e0 + e1 * e1 + e2 * e2 +
                 0.5 * ((G[0][1] + G[1][0]) * (G[0][1] + G[1][0]) + (G[1][2] + G[2][1]) * (G[1][2] + G[2][1]) +
                        (G[0][2] + G[2][0]) * (G[0][2] + G[2][0]));
        else
            ss = e0 * e0 + e1 * e1 + 0.5 * (G[0][1] + G[1][0]) * (G[0][1] + G[1][0]);
        const double gnorm = sqrt(2.0 * ss) * ir0;
        if (closure == CL_POWERLAW) {
            tau_i = 0.5 + a.pl_k3 * pow(gnorm, a.pl_nm1);
            if (!(tau_i >= a.pl_tau_min)) tau_i = a.pl_tau_min;
            if (tau_i > a.pl_tau_max) tau_i = a.pl_tau_max;
        } else {
            tau_i = a.tau0 + a.smag_c3 * gnorm;
        }
    }
    if (tau_field) tau_field[node] = R(tau_i);
    if (gu) {
        const double snu = closure == CL_NEWTON ? double(a.s[L::NU0]) : 1.0 / tau_i;
        const double divj = G[0][0] + G[1][1] + G[2][2];
        if constexpr (Q == 19) {
            mn[1] = -38.0 / (3.0 * a.s[1]) * divj;
            mn[9] = -2.0 / (3.0 * snu) * (3.0 * G[0][0] - divj);
            mn[11] = -2.0 / (3.0 * snu) * (G[1][1] - G[2][2]);
            mn[13] = -(G[1][0] + G[0][1]) / (3.0 * snu);
            mn[14] = -(G[2][1] + G[1][2]) / (3.0 * snu);
            mn[15] = -(G[0][2] + G[2][0]) / (3.0 * snu);
        } else if constexpr (Q == 15) {
            mn[1] = -2.0 / (3.0 * a.s[1]) * divj;
            mn[9] = -2.0 / (3.0 * snu) * (3.0 * G[0][0] - divj);
            mn[10] = -2.0 / (3.0 * snu) * (G[1][1] - G[2][2]);
            mn[11] = -(G[1][0] + G[0][1]) / (3.0 * snu);
            mn[12] = -(G[2][1] + G[1][2]) / (3.0 * snu);
            mn[13] = -(G[0][2] + G[2][0]) / (3.0 * snu);
        } else {
            mn[1] = -2.0 * divj / a.s[1];
            mn[7] = -2.0 * (G[0][0] - G[1][1]) / (3.0 * snu);
            mn[8] = -(G[1][0] + G[0][1]) / (3.0 * snu);
        }
    }
    double Dk[Q], add[Q];
    sfor<Q>([&](auto k) { Dk[k] = mn[k] * (1.0 / norm2<L>(CV(k))); });
    back_transform<L, (1u << Q) - 1u>(Dk, add);
    const double jj = (j[0] * j[0] + j[1] * j[1] + j[2] * j[2]) * ir0;
    const double jF = (j[0] * F[0] + j[1] * F[1] + j[2] * F[2]) * ir0;
    ST* __restrict__ buf = static_cast<ST*>(a.dst);
    const int dims[3] = {nx, ny, nz};
    const int pos[3] = {x, y, z};
    sfor<Q>([&](auto i) {
        constexpr int cx = L::c(CV(i), 0), cy = L::c(CV(i), 1), cz = L::c(CV(i), 2);
        const double w = double(L::wnum(CV(i))) / L::WDEN;
        const double cj = cx * j[0] + cy * j[1] + cz * j[2];
        const double cF = cx * F[0] + cy * F[1] + cz * F[2];
        const double feq = w * (dr + 3.0 * cj + 4.5 * cj * cj * ir0 - 1.5 * jj);
        const double fb = w * (3.0 * cF - 3.0 * jF + 9.0 * cj * cF * ir0);
        double v = feq + add[i] - 0.5 * fb;
        // un-stream: write where the pull of (node, i) will read
        int s[3];
        int nout = 0, face = -1;
        for (int ax = 0; ax < 3; ++ax) {
            const int cax = ax == 0 ? cx : (ax == 1 ? cy : cz);
            s[ax] = pos[ax] - cax;
            if (cax == 0 || (s[ax] >= 0 && s[ax] < dims[ax])) continue;
            const int fc = 2 * ax + (s[ax] < 0 ? 0 : 1);
            if ((a.wall_mask >> fc) & 1) {
                ++nout;
                face = fc;
            } else {
                s[ax] = s[ax] < 0 ? s[ax] + dims[ax] : s[ax] - dims[ax];
            }
        }
        if (nout == 0) {
            Store<ST>::st(buf + CV(i) * a.stride + (s[2] * ny + s[1]) * nx + s[0], R(v));
        } else {
            if (nout == 1 && ((a.lid_mask >> face) & 1)) {
                const double cu = cx * a.lid[face][0] + cy * a.lid[face][1] + cz * a.lid[face][2];
                v -= 6.0 * w * r0 * cu;
            }
            Store<ST>::st(buf + opp<L>(CV(i)) * a.stride + node, R(v));
        }
    });
}

// ------------------------------------------------------------------------------------------
// global sums: each block walks whole rows (fixed assignment, so the result is reproducible);
// each node's totals are formed in the compute type, then FP32 states accumulate them across nodes
// with an error-free two-sum (hi, lo) pair per component, FP64 states in plain FP64; per-block
// partials go to scratch as FP64 and one ordered pass adds them.

constexpr int SUM_THREADS = 256;

template <class R>
struct Comp {
    R hi = R(0), lo = R(0);
    __device__ __forceinline__ void add(R x) {
        if constexpr (sizeof(R) == 4) {
            const R t = hi + x;
            const R bp = t - hi;
            lo += (hi - (t - bp)) + (x - bp);
            hi = t;
        } else {
            hi += x;
        }
    }
    __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

template <class L, class ST>
__global__ void __launch_bounds__(SUM_THREADS) k_sums(const StepArgs<typename Store<ST>::R> a, double* __restrict__ partial) {
    using R = typename Store<ST>::R;
    constexpr int D = L::D;
    const long long N = (long long)a.nx * a.ny * a.nz;  // component offsets c*N exceed 2^31 on big grids
    const int rows = a.ny * a.nzc;  // the computed planes only (a halo plane belongs to a neighbour)
    Comp<R> acc[1 + D];
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int y = r % a.ny, z = r / a.ny + a.z0;
        for (int x = threadIdx.x; x < a.nx; x += blockDim.x) {
            R f[L::Q];
            pull<L, ST>(a, x, y, z, f);
            // the node's own totals in plain arithmetic (19 values of one node), then one
            // compensated add per component across nodes
            R m0 = nzero<R>(), mj[3] = {nzero<R>(), nzero<R>(), nzero<R>()};
            sfor<L::Q>([&](auto i) {
                m0 += f[i];
                sfor<D>([&](auto d) { mj[d] = cadd<L::c(CV(i), CV(d))>(mj[d], f[i]); });
            });
            const int n = (z * a.ny + y) * a.nx + x;
            acc[0].add(m0);
#pragma unroll
            for (int d = 0; d < D; ++d)
                acc[1 + d].add(fma(R(0.5), a.force_field ? a.force_field[d * N + n] : a.F[d], mj[d]));
        }
    }
    __shared__ double red[SUM_THREADS / 32][1 + D];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c <= D; ++c) {
        double v = acc[c].value();
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c <= D; ++c) {
            double v = 0.0;
            for (int w = 0; w < SUM_THREADS / 32; ++w) v += red[w][c];
            partial[blockIdx.x * (1 + D) + c] = v;
        }
    }
}

// sums nblocks partial rows of width `width` in block order into out[width]
__global__ void k_sums_final(const double* __restrict__ partial, int nblocks, int width, double* __restrict__ out);

}  // namespace lbm
