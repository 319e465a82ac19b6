// step_pair.cuh -- the step of two x-adjacent nodes per thread in packed FP32-pair arithmetic
// (16-bit storage).
//
// The 16-bit step moves half the bytes of the FP32 step but executes the same FP32 collision, so
// per node it is bound by instruction issue, not by HBM.  A thread here owns two x-adjacent nodes:
// they share the pull's address arithmetic (pull2: one paired load where c_x = 0), and their
// collisions run side by side as one pair of FP32 lanes, each add, multiply and fused multiply-add
// acting on both lanes with one instruction (add/mul/fma.rn.f32x2; round to nearest in each lane,
// as the scalar operations round).  The moment transforms, the equilibrium and force moments,
// Chai's non-equilibrium distributions and the strain contractions are the generic code of
// step.cuh instantiated on the pair type; the closure's fixed point runs lane by lane, so each node
// stops after its own sweeps.
//
// Holding two nodes' values doubles the live state, so the post-collision populations are formed
// from moments, f*_i = sum_k T_ki G_k with G_k = m*_k / |T_k|^2 (eq. (mrteqvT) with the orthogonal
// basis: T^-1 = T^t diag(1/|T_k|^2)), instead of the one-node kernels' delta form f* = f - T^-1(...):
// the pulled populations then die after the forward transform.  The FP32 rounding of the moment
// form is far below the 16-bit storage's (2^-11 relative for FP16, 2^-8 for BF16), and both nodes'
// results leave with one 32-bit store per population.
#pragma once

#include "step.cuh"

namespace lbm {

// two lanes of FP32, one per node
struct V2 {
    float2 v;
    V2() = default;
    __device__ __forceinline__ V2(float s) : v{s, s} {}  // the same value in both lanes
    __device__ __forceinline__ V2(float a, float b) : v{a, b} {}
    __device__ __forceinline__ explicit V2(float2 u) : v(u) {}
    __device__ __forceinline__ float lo() const { return v.x; }
    __device__ __forceinline__ float hi() const { return v.y; }
};
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return V2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ V2 operator-(V2 a) { return V2(-a.v.x, -a.v.y); }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return V2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))); }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return V2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ V2& operator+=(V2& a, V2 b) { return a = a + b; }
__device__ __forceinline__ V2& operator-=(V2& a, V2 b) { return a = a - b; }
__device__ __forceinline__ V2 fma(V2 a, V2 b, V2 c) { return V2(__ffma2_rn(a.v, b.v, c.v)); }

// Smagorinsky / Newtonian closure for the pair: the quadratic form of |S|^2 in s = 1/tau is formed
// for both lanes at once, then each lane runs the scalar fixed point of step.cuh.
template <class L, int CLOSURE>
__device__ __forceinline__ V2 solve_tau_pair(const V2 (&A)[L::NS], const V2 (&B)[L::NS], const StepArgs<float>& a,
                                            V2& snu) {
    static_assert(CLOSURE == CL_NEWTON || CLOSURE == CL_SMAG, "16-bit storage builds these closures");
    if constexpr (CLOSURE == CL_NEWTON) {
        snu = V2(a.s[L::NU0]);
        return V2(a.tau0);
    } else {
        const V2 qa = strain_dot<L>(A, A), qb2 = V2(2.0f) * strain_dot<L>(A, B), qc = strain_dot<L>(B, B);
        const float t0 = tau_fixed_point<CLOSURE>(qa.lo(), qb2.lo(), qc.lo(), a);
        const float t1 = tau_fixed_point<CLOSURE>(qa.hi(), qb2.hi(), qc.hi(), a);
        snu = V2(c_rcp(t0), c_rcp(t1));
        return V2(t0, t1);
    }
}

// One step of the pair (node, node + 1) from its pulled populations: the step_body arithmetic on
// pairs, then one paired store per population.  node is even, so every pair is 4-byte aligned
// (and the force field's pair 8-byte aligned).
template <class L, class ST, int CLOSURE, int FORMULA, bool FORCE>
__device__ __forceinline__ void step_pair(const StepArgs<float>& a, const F2 (&f2)[L::Q], int node) {
    using R = V2;
    constexpr int Q = L::Q, NS = L::NS, NP = L::NP;
    const long long N = (long long)a.nx * a.ny * a.nz;

    R f[Q];
    sfor<Q>([&](auto i) { f[i] = V2(f2[i].v); });
    R P[NP], Dd[NP];
    sfor<NP>([&](auto p) {
        P[p] = f[L::pa(CV(p))] + f[L::pb(CV(p))];
        Dd[p] = f[L::pa(CV(p))] - f[L::pb(CV(p))];
    });
    R F[3] = {R(0.0f), R(0.0f), R(0.0f)};
    if constexpr (FORCE) {
        if (a.force_field) {
            sfor<L::D>([&](auto d) {
                F[d] = V2(ld2_keep(a.force_field + CV(d) * N + node));
            });
        } else {
            sfor<L::D>([&](auto d) { F[d] = R(a.F[d]); });
        }
    }
    const R ir0 = R(a.inv_rho0);
    R drho, j[3] = {R(0.0f), R(0.0f), R(0.0f)}, u[3] = {R(0.0f), R(0.0f), R(0.0f)};
    R snu;
    R G[Q];  // f*_i = sum_k T_ki G_k

    if constexpr (FORMULA == F_YU) {
        // f* = T^-1 m* written as f*_i = sum_k T_ki G_k with G_k = m_k / |T_k|^2 - D_k (the basis is
        // orthogonal), so the pulled populations are not needed after the forward transform: the
        // G_k of the rate-independent moments are final before the closure, the viscous ones keep
        // m_k / |T_k|^2 - (force part) and mn_k until the closure gives s_nu.
        R m[Q];
        Xf<L>::forward(f[0], P, Dd, m);
        drho = m[0];
        j[0] = FORCE ? fma(R(0.5f), F[0], m[3]) : m[3];
        j[1] = FORCE ? fma(R(0.5f), F[1], m[5]) : m[5];
        if constexpr (L::D == 3) j[2] = FORCE ? fma(R(0.5f), F[2], m[7]) : m[7];
        sfor<L::D>([&](auto d) { u[d] = j[d] * ir0; });
        R mn[Q];
        {
            R meq[Q], TF[Q];
            Eq<L>::meq(drho, j, u, meq);
            if constexpr (FORCE) Eq<L>::tforce(u, F, TF);
            sfor<Q>([&](auto k) {
                constexpr double inv_n = 1.0 / norm2<L>(CV(k));
                const bool has_tf = FORCE && !Eq<L>::ghost(CV(k)) && CV(k) != 0;
                if constexpr (L::conserved(CV(k))) {
                    mn[k] = R(0.0f);
                    // D_k = -TF_k / |T_k|^2
                    if constexpr (has_tf)
                        G[k] = cst<R>(inv_n) * (m[k] + TF[k]);
                    else
                        G[k] = cst<R>(inv_n) * m[k];
                } else {
                    if constexpr (Eq<L>::ghost(CV(k)))
                        mn[k] = m[k];
                    else if constexpr (FORCE)
                        mn[k] = fma(R(0.5f), TF[k], m[k] - meq[k]);
                    else
                        mn[k] = m[k] - meq[k];
                    // the rate-independent part of G_k: (m_k + TF_k) / |T_k|^2, less s_k mn_k / |T_k|^2
                    // unless k is viscous
                    const R base = has_tf ? cst<R>(inv_n) * (m[k] + TF[k]) : cst<R>(inv_n) * m[k];
                    if constexpr (L::viscous(CV(k)))
                        G[k] = base;
                    else
                        G[k] = fma(R(-a.skn[k]), mn[k], base);
                }
            });
        }
        R A[NS], B[NS];
        Eq<L>::yu_split(mn, R(a.s[1] * float(Eq<L>::YU_A)) * ir0, ir0, A, B);
        solve_tau_pair<L, CLOSURE>(A, B, a, snu);
        sfor<Q>([&](auto k) {
            if constexpr (L::viscous(CV(k))) {
                constexpr double inv_n = 1.0 / norm2<L>(CV(k));
                G[k] = fma(-(snu * cst<R>(inv_n)), mn[k], G[k]);
            }
        });
    } else {
        // Chai route: the non-equilibrium distributions f - f_eq + Fbar/2 (opposite-pair form), their
        // moments mn = T fn, Omega = T^-1 L mn back in distribution space (even parts: only those
        // enter the contraction) and S = -N / (2 rho0 cs^2) with N = sum_i c_i c_i Omega_i.  The
        // post-collision state is then formed from the same mn as f* = T^-1 m*, m*_k = m_eq_k +
        // TF_k/2 + (1 - s_k) mn_k (the moments of f are mn + m_eq - TF/2), so neither f nor fn has to
        // stay live across the transforms.
        drho = f[0];
        sfor<NP>([&](auto p) { drho += P[p]; });
        sfor<L::D>([&](auto d) {
            R acc = nzero<R>();
            sfor<NP>([&](auto p) { acc = cadd<L::c(L::pa(CV(p)), CV(d))>(acc, Dd[p]); });
            j[d] = FORCE ? fma(R(0.5f), F[d], acc) : acc;
            u[d] = j[d] * ir0;
        });
        R mn[Q];
        {
            R fn0, Pn[NP], Dn[NP];
            noneq_pairs<L, FORCE>(f[0], P, Dd, drho, j, u, F, fn0, Pn, Dn);
            Xf<L>::forward(fn0, Pn, Dn, mn);
        }
        const R kS = R(-1.5f) * ir0;
        if constexpr (CLOSURE == CL_NEWTON) {
            snu = R(a.s[L::NU0]);  // with fixed rates S is a read-out only, not needed by the step
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
            solve_tau_pair<L, CLOSURE>(A, B, a, snu);
        }
        {
            R meq[Q], TF[Q];
            Eq<L>::meq(drho, j, u, meq);
            if constexpr (FORCE) Eq<L>::tforce(u, F, TF);
            sfor<Q>([&](auto k) {
                constexpr double inv_n = 1.0 / norm2<L>(CV(k));
                const bool has_tf = FORCE && !Eq<L>::ghost(CV(k)) && CV(k) != 0;
                // m_k + TF_k = mn_k + m_eq_k + TF_k / 2
                R base = Eq<L>::ghost(CV(k)) ? mn[k] : mn[k] + meq[k];
                if constexpr (has_tf) base = fma(R(0.5f), TF[k], base);
                base = cst<R>(inv_n) * base;
                if constexpr (L::conserved(CV(k)))
                    G[k] = base;
                else if constexpr (L::viscous(CV(k)))
                    G[k] = fma(-(snu * cst<R>(inv_n)), mn[k], base);
                else
                    G[k] = fma(R(-a.skn[k]), mn[k], base);
            });
        }
    }
    R fs[Q];
    Xf<L>::template backward<mask_all<L>()>(G, fs);
    sfor<Q>([&](auto i) { Store<ST>::st2(static_cast<ST*>(a.dstp[CV(i)]) + node, fs[i].lo(), fs[i].hi()); });
}

// Two x-adjacent nodes per thread (16-bit storage, nx even).  Bound to 7 resident blocks per SM
// (72 registers) for both routes: measured on a GB300 against 8 blocks (Yu: channel -4%, 512^3 box
// +1%) and, for the Chai route, 6 and 5 blocks (80 and 96 registers, fewer spilled values: channel
// FP16 40.6 and 43.4 against 45.4 GLUPS, 512^3 box within 1%).
constexpr int PAIR_MIN_BLOCKS = 7;

template <class L, class ST, int CLOSURE, int FORMULA, bool FORCE>
__global__ void __launch_bounds__(128, PAIR_MIN_BLOCKS) k_step_pair_seq(const StepArgs<typename Store<ST>::R> a) {
    pdl_wait();
    pdl_release();
    const int x = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z + a.z0;
    if (x >= a.nx || y >= a.ny) return;
    F2 f2[L::Q];
    pull2<L, ST>(a, x, y, z, f2);
    step_pair<L, ST, CLOSURE, FORMULA, FORCE>(a, f2, (z * a.ny + y) * a.nx + x);
}

}  // namespace lbm
