// adjoint.cuh -- reverse-mode derivative of the fused D3Q19 MRT step with the Smagorinsky
// closure, with respect to a body-force field, and of the dissipation functional
//   L = sum_x nu_eff(x) sum_ab S_ab(x)^2,  nu_eff = (tau - 1/2)/3,
// evaluated on the pre-collision state the step after the last one would see.
//
// Forward map of one node (pulled populations p, force density F = rho0 g at the node):
//   m = T p, drho = m0, j = (m3, m5, m7) + F/2, m_eq(drho, j) (eq. (meq)), TF = J(j) F with
//   J = d m_eq / d j, mn = m - m_eq + TF/2 (non-conserved moments), S = A(mn) + s B(mn) (Yu's
//   formula, eq. (LuoS)), tau = tau0 + 3 Cs^2 |S| solved as a fixed point, s = 1/tau,
//   D_k = (s_k mn_k - TF_k)/|T_k|^2, f* = p - T^T D.
// Reverse map for an adjoint lambda = dL/df* at the node (and optional direct adjoints of S and
// tau, used by the functional): D' = -T lambda; s' = sum_visc D'_k mn_k/|T_k|^2 + S'.B;
// tau' = tau'_direct - s' s^2; the closure is differentiated at its converged fixed point
// (implicit function rule; |S| = 0 contributes nothing); mn' = Y^T(sigma) + D'_k s_k/|T_k|^2 with
// sigma = S' + tau' 3Cs^2 (2 w S/|S|)/(1 + 3Cs^2 s^2 2 (w S).B/|S|); TF' = -D'/|T|^2 + mn'/2;
// m_eq' = -mn'; drho' = -11 m_eq'_1 + 3 m_eq'_2; j' = J^T m_eq' + sum_k TF'_k H_k F (H_k the
// constant Hessian of m_eq_k in j); F' = J^T TF' + j'/2; p' = lambda + T^T (drho', ..., j', mn').
// Both strain routes compute the same function (Sec. 5.1), so one derivative serves both.
//
// Adjoint streaming: p_i(x) = f_i(x - c_i), so lambda_n,i(y) = mu_i(y + c_i) where mu = p' of
// the node: each node writes its mu_i back to the source x - c_i of its pull (periodic wrap).
#pragma once

#include "step.cuh"
#include "step_stream.cuh"

namespace lbm {

// the quantities of the node's forward map that the reverse map needs
template <class R>
struct NodeFwd {
    R mn[19];
    R j[3], F[3];
    R S[6], B[6];
    R tau, s, snorm;
};

template <class R>
__device__ __forceinline__ R strain_w_dot(const R (&S)[6], const R (&T)[6]) {
    return S[0] * T[0] + S[1] * T[1] + S[2] * T[2] + R(2) * (S[3] * T[3] + S[4] * T[4] + S[5] * T[5]);
}

// J(jv)^T v for the 19-vector v (only entries 1..15 enter), J = d m_eq / d j at j = jv
template <class R>
__device__ __forceinline__ void jt(const R (&jv)[3], const R (&v)[19], R ir0, R (&out)[3]) {
    const R a9 = v[9] - R(0.5) * v[10], a11 = v[11] - R(0.5) * v[12];
    const R e = R(38) * v[1] - R(11) * v[2];
    out[0] = ir0 * (e * jv[0] + R(4) * jv[0] * a9 + jv[1] * v[13] + jv[2] * v[15]) + v[3] - cst<R>(2.0 / 3.0) * v[4];
    out[1] = ir0 * (e * jv[1] - R(2) * jv[1] * a9 + R(2) * jv[1] * a11 + jv[0] * v[13] + jv[2] * v[14]) + v[5] -
             cst<R>(2.0 / 3.0) * v[6];
    out[2] = ir0 * (e * jv[2] - R(2) * jv[2] * a9 - R(2) * jv[2] * a11 + jv[1] * v[14] + jv[0] * v[15]) + v[7] -
             cst<R>(2.0 / 3.0) * v[8];
}

// forward map of one node (Yu form, Smagorinsky or Newtonian closure)
template <int CLOSURE, class R>
__device__ __forceinline__ void node_forward(const R (&p)[19], const R (&F)[3], const StepArgs<R>& a, NodeFwd<R>& st) {
    R P[9], Dd[9], m[19];
    sfor<9>([&](auto q) {
        P[q] = p[D3Q19::pa(CV(q))] + p[D3Q19::pb(CV(q))];
        Dd[q] = p[D3Q19::pa(CV(q))] - p[D3Q19::pb(CV(q))];
    });
    Xf<D3Q19>::forward(p[0], P, Dd, m);
    const R ir0 = a.inv_rho0;
    R u[3], meq[19], TF[19];
    st.j[0] = fma(R(0.5), F[0], m[3]);
    st.j[1] = fma(R(0.5), F[1], m[5]);
    st.j[2] = fma(R(0.5), F[2], m[7]);
    for (int d = 0; d < 3; ++d) {
        u[d] = st.j[d] * ir0;
        st.F[d] = F[d];
    }
    Eq<D3Q19>::meq(m[0], st.j, u, meq);
    Eq<D3Q19>::tforce(u, F, TF);
    sfor<19>([&](auto k) {
        if constexpr (D3Q19::conserved(CV(k)))
            st.mn[k] = R(0);
        else
            st.mn[k] = fma(R(0.5), TF[k], m[k] - meq[k]);
    });
    R A[6];
    Eq<D3Q19>::yu_split(st.mn, a.s[1] * R(Eq<D3Q19>::YU_A) * ir0, ir0, A, st.B);
    st.tau = solve_tau<D3Q19, R, CLOSURE>(A, st.B, a, st.S, st.s, 0);  // Newtonian / Smagorinsky only
    st.snorm = sqrt(R(2) * strain_w_dot(st.S, st.S));
}

// Reverse map of one node.  lam: adjoint of f* (ignored when HAS_LAM is false); Sbar, taubar_d:
// direct adjoints of S and tau.  Outputs mu = dL/dp and Fbar = dL/dF at the node.
template <int CLOSURE, bool HAS_LAM, class R>
__device__ __forceinline__ void node_backward(const NodeFwd<R>& st, const R (&lam)[19], const R (&Sbar)[6], R taubar_d,
                                              const StepArgs<R>& a, R (&mu)[19], R (&Fbar)[3]) {
    const R ir0 = a.inv_rho0;
    R Db[19];  // D' = -T lam
    if constexpr (HAS_LAM) {
        R P[9], Dd[9], Lm[19];
        sfor<9>([&](auto q) {
            P[q] = lam[D3Q19::pa(CV(q))] + lam[D3Q19::pb(CV(q))];
            Dd[q] = lam[D3Q19::pa(CV(q))] - lam[D3Q19::pb(CV(q))];
        });
        Xf<D3Q19>::forward(lam[0], P, Dd, Lm);
        sfor<19>([&](auto k) { Db[k] = -Lm[k]; });
    } else {
        sfor<19>([&](auto k) { Db[k] = R(0); });
    }
    // s' and tau'
    R sbar = Sbar[0] * st.B[0] + Sbar[1] * st.B[1] + Sbar[2] * st.B[2] + Sbar[3] * st.B[3] + Sbar[4] * st.B[4] +
             Sbar[5] * st.B[5];
    sfor<19>([&](auto k) {
        if constexpr (D3Q19::viscous(CV(k))) sbar = fma(Db[k] * cst<R>(1.0 / norm2<D3Q19>(CV(k))), st.mn[k], sbar);
    });
    R sig[6];
    sfor<6>([&](auto c) { sig[c] = Sbar[c]; });
    if constexpr (CLOSURE != CL_NEWTON) {
        const R taubar = taubar_d - sbar * st.s * st.s;
        if (st.snorm > R(0)) {
            const R c3 = a.smag_c3;
            const R SB = strain_w_dot(st.S, st.B);
            const R den = R(1) + R(2) * c3 * st.s * st.s * SB / st.snorm;
            const R coef = taubar * c3 * R(2) / (st.snorm * den);
            sfor<6>([&](auto c) { sig[c] = fma(coef * R(CV(c) < 3 ? 1 : 2), st.S[c], sig[c]); });
        }
    }
    // mn' = Y^T(sigma) + D'_k s_k / |T_k|^2
    R mnb[19];
    sfor<19>([&](auto k) { mnb[k] = R(0); });
    mnb[1] = -(a.s[1] * R(Eq<D3Q19>::YU_A) * ir0) * (sig[0] + sig[1] + sig[2]);
    mnb[9] = st.s * ir0 * (R(-0.5) * sig[0] + R(0.25) * (sig[1] + sig[2]));
    mnb[11] = st.s * ir0 * (R(0.75) * (sig[2] - sig[1]));
    mnb[13] = st.s * ir0 * (R(-1.5) * sig[3]);
    mnb[14] = st.s * ir0 * (R(-1.5) * sig[4]);
    mnb[15] = st.s * ir0 * (R(-1.5) * sig[5]);
    sfor<19>([&](auto k) {
        if constexpr (!D3Q19::conserved(CV(k))) {
            const R sk = D3Q19::viscous(CV(k)) ? st.s * cst<R>(1.0 / norm2<D3Q19>(CV(k))) : R(a.skn[k]);
            mnb[k] = fma(Db[k], sk, mnb[k]);
        }
    });
    // TF' and m_eq'
    R TFb[19], meqb[19];
    sfor<19>([&](auto k) {
        constexpr double inv_n = 1.0 / norm2<D3Q19>(CV(k));
        if constexpr (D3Q19::conserved(CV(k)))
            TFb[k] = cst<R>(-inv_n) * Db[k];
        else
            TFb[k] = fma(R(0.5), mnb[k], cst<R>(-inv_n) * Db[k]);
        meqb[k] = -mnb[k];
    });
    // j' = J^T m_eq' + sum_k TF'_k H_k F ;  F' = J^T TF' + j'/2
    R jb[3], hF[3], jtf[3];
    jt(st.j, meqb, ir0, jb);
    {
        // sum_k TF'_k H_k F = (J(F)^T TF') - (the j-independent rows 3..8 of J)^T TF'
        jt(st.F, TFb, ir0, hF);
        hF[0] -= TFb[3] - cst<R>(2.0 / 3.0) * TFb[4];
        hF[1] -= TFb[5] - cst<R>(2.0 / 3.0) * TFb[6];
        hF[2] -= TFb[7] - cst<R>(2.0 / 3.0) * TFb[8];
    }
    jt(st.j, TFb, ir0, jtf);
    for (int d = 0; d < 3; ++d) {
        jb[d] += hF[d];
        Fbar[d] = fma(R(0.5), jb[d], jtf[d]);
    }
    // m' and p' = lam + T^T m'
    R mb[19];
    sfor<19>([&](auto k) { mb[k] = mnb[k]; });
    mb[3] = jb[0];
    mb[5] = jb[1];
    mb[7] = jb[2];
    const R drhob = R(-11) * meqb[1] + R(3) * meqb[2];
    R back[19];
    Xf<D3Q19>::template backward<mask_all_but_density<D3Q19>()>(mb, back);
    sfor<19>([&](auto i) {
        if constexpr (HAS_LAM)
            mu[i] = lam[i] + (back[i] + drhob);
        else
            mu[i] = back[i] + drhob;
    });
}

// ------------------------------------------------------------------------------------------
// kernels (periodic box; force field required)

template <class R>
struct AdjArgs {
    StepArgs<R> st;      // lattice, rates, closure, force field; srcp = the state f^n
    const R* lam_in;     // lambda_{n+1}, q arrays of `stride` (step) or unused (functional)
    R* lam_out;          // lambda_n
    const R* lamp_in[19];  // lam_in + i * stride (filled on the host, see set_lambda)
    R* lamp_out[19];       // lam_out + i * stride
    R* dF;               // 3 x N accumulator of dL/dF over the current segment
    double* partial;     // functional: one FP64 partial sum per block
};

// host side: the lambda buffers and their per-population base pointers
template <class R>
inline void set_lambda(AdjArgs<R>* a, const R* in, R* out) {
    a->lam_in = in;
    a->lam_out = out;
    for (int i = 0; i < 19; ++i) {
        a->lamp_in[i] = in ? in + i * a->st.stride : nullptr;
        a->lamp_out[i] = out ? out + i * a->st.stride : nullptr;
    }
}

// write mu_i to the pull's source node x - c_i (periodic): the transpose of the pull.  Nodes away
// from every face write at node - c_i (a warp-uniform offset); the others wrap by index.
template <class R>
__device__ __forceinline__ void push(const AdjArgs<R>& a, int x, int y, int z, const R (&mu)[19]) {
    const int nx = a.st.nx, ny = a.st.ny, nz = a.st.nz, nxy = nx * ny;
    const int node = (z * ny + y) * nx + x;
    if (x > 0 && x < nx - 1 && y > 0 && y < ny - 1 && z > 0 && z < nz - 1) {
        sfor<19>([&](auto i) {
            constexpr int cx = D3Q19::c(CV(i), 0), cy = D3Q19::c(CV(i), 1), cz = D3Q19::c(CV(i), 2);
            a.lamp_out[CV(i)][node - (cx + cy * nx + cz * nxy)] = mu[i];
        });
        return;
    }
    sfor<19>([&](auto i) {
        constexpr int cx = D3Q19::c(CV(i), 0), cy = D3Q19::c(CV(i), 1), cz = D3Q19::c(CV(i), 2);
        int tx = x - cx, ty = y - cy, tz = z - cz;
        tx = tx < 0 ? tx + nx : (tx >= nx ? tx - nx : tx);
        ty = ty < 0 ? ty + ny : (ty >= ny ? ty - ny : ty);
        tz = tz < 0 ? tz + nz : (tz >= nz ? tz - nz : tz);
        a.lamp_out[CV(i)][(tz * ny + ty) * nx + tx] = mu[i];
    });
}

template <class ST>
struct AdjTypes {
    using R = typename Store<ST>::R;
};

// one adjoint step: lambda_n = Push(mu(p^n, lambda_{n+1})), dF += F'
template <class ST, int CLOSURE>
__global__ void __launch_bounds__(128) k_adjoint_step(const AdjArgs<typename Store<ST>::R> a) {
    using R = typename Store<ST>::R;
    pdl_wait();     // lambda_{n+1} and the recomputed state are complete and visible from here on
    pdl_release();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= a.st.nx || y >= a.st.ny) return;
    const long long N = (long long)a.st.nx * a.st.ny * a.st.nz;  // component offsets d*N exceed 2^31
    const int node = (z * a.st.ny + y) * a.st.nx + x;
    R p[19], F[3], lam[19], acc[3];
    pull<D3Q19, ST>(a.st, x, y, z, p);
    for (int d = 0; d < 3; ++d) F[d] = ld_keep(a.st.force_field + d * N + node);
    sfor<19>([&](auto i) { lam[i] = a.lamp_in[CV(i)][node]; });
    // the node's force-gradient accumulator, loaded with the other inputs (its latency overlaps
    // theirs instead of following the reverse map)
    for (int d = 0; d < 3; ++d) acc[d] = load_early(a.dF + d * N + node);
    NodeFwd<R> st;
    node_forward<CLOSURE>(p, F, a.st, st);
    R mu[19], Fb[3];
    const R Sb[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    node_backward<CLOSURE, true>(st, lam, Sb, R(0), a.st, mu, Fb);
    push(a, x, y, z, mu);
    for (int d = 0; d < 3; ++d) a.dF[d * N + node] = acc[d] + Fb[d];
}

// Several adjoint steps in one launch (the scheduler of step_stream.cuh): launch step k is the
// reverse step of the state a0.st's source shifted by -k * c.ring elements (the states of a
// checkpoint segment, equally spaced, visited backwards); lambda ping-pongs, a0 reading the first
// lambda buffer and writing the second, a1 the reverse.  The nine-unit dependency covers the
// push: step k writes lambda entries of the neighbouring units, which read their own entries of
// step k - 1's output and wrote the buffer's previous contents.  lambda and the force-gradient
// accumulator, which other blocks of the launch wrote, are read through L2; the states are
// read-only for the whole launch.
template <class ST, int CLOSURE>
__device__ __forceinline__ void adjoint_unit(const AdjArgs<typename Store<ST>::R>& a, int z, int y0, int y1,
                                             long long es) {
    using R = typename Store<ST>::R;
    const long long N = (long long)a.st.nx * a.st.ny * a.st.nz;
    for (int y = y0; y < y1; ++y) {
        for (int x = threadIdx.x; x < a.st.nx; x += blockDim.x) {
            const int node = (z * a.st.ny + y) * a.st.nx + x;
            R p[19], F[3], lam[19], acc[3];
            pull<D3Q19, ST>(a.st, x, y, z, p, es);
            for (int d = 0; d < 3; ++d) F[d] = ld_keep(a.st.force_field + d * N + node);
            sfor<19>([&](auto i) { lam[i] = __ldcg(a.lamp_in[CV(i)] + node); });
            // the accumulator (this node's own, last written by this unit's previous step, which
            // the unit's dependencies include) loaded with the other inputs
            for (int d = 0; d < 3; ++d) acc[d] = load_early(a.dF + d * N + node);
            NodeFwd<R> st;
            node_forward<CLOSURE>(p, F, a.st, st);
            R mu[19], Fb[3];
            const R Sb[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
            node_backward<CLOSURE, true>(st, lam, Sb, R(0), a.st, mu, Fb);
            push(a, x, y, z, mu);
            for (int d = 0; d < 3; ++d) a.dF[d * N + node] = acc[d] + Fb[d];
        }
    }
}

// Bound to 8 resident blocks per SM (64 registers, a few spilled values): measured faster than 7
// blocks at 72 registers and than 6 at 80 (the reverse step waits on memory; more warps hide it).
template <class ST, int CLOSURE>
__global__ void __launch_bounds__(128, 8) k_adjoint_stream(const AdjArgs<typename Store<ST>::R> a0,
                                                        const AdjArgs<typename Store<ST>::R> a1, const StreamCtl c) {
    stream_schedule(a0.st.ny, a0.st.nz, c, [&](int k, int z, int y0, int y1) {
        const long long es = -(long long)k * c.ring;
        if (k & 1)
            adjoint_unit<ST, CLOSURE>(a1, z, y0, y1, es);
        else
            adjoint_unit<ST, CLOSURE>(a0, z, y0, y1, es);
    });
}

// the functional at the final state: per-block FP64 partial sums of nu_eff S:S, the adjoint
// lambda_T = Push(dL/dp), and dF initialised to the functional's direct dL/dF
template <class ST, int CLOSURE>
__global__ void __launch_bounds__(128) k_functional(const AdjArgs<typename Store<ST>::R> a) {
    using R = typename Store<ST>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const bool active = x < a.st.nx && y < a.st.ny;
    double ell = 0.0;
    if (active) {
        const long long N = (long long)a.st.nx * a.st.ny * a.st.nz;  // component offsets d*N exceed 2^31
        const int node = (z * a.st.ny + y) * a.st.nx + x;
        R p[19], F[3];
        pull<D3Q19, ST>(a.st, x, y, z, p);
        for (int d = 0; d < 3; ++d) F[d] = ld_keep(a.st.force_field + d * N + node);
        NodeFwd<R> st;
        node_forward<CLOSURE>(p, F, a.st, st);
        const R nu = (st.tau - R(0.5)) * cst<R>(1.0 / 3.0);
        const R SS = strain_w_dot(st.S, st.S);
        ell = double(nu * SS);
        R Sb[6];
        sfor<6>([&](auto c) { Sb[c] = R(2) * nu * R(CV(c) < 3 ? 1 : 2) * st.S[c]; });
        R mu[19], Fb[3];
        const R none[19] = {};
        node_backward<CLOSURE, false>(st, none, Sb, SS * cst<R>(1.0 / 3.0), a.st, mu, Fb);
        push(a, x, y, z, mu);
        for (int d = 0; d < 3; ++d) a.dF[d * N + node] = Fb[d];
    }
    // block sum of ell in FP64 (fixed order: warp tree, then warps in order)
    __shared__ double red[4];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) ell += __shfl_down_sync(0xffffffffu, ell, o);
    if ((t & 31) == 0) red[t >> 5] = ell;
    __syncthreads();
    if (t == 0) {
        const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        a.partial[b] = red[0] + red[1] + red[2] + red[3];
    }
}

// dLdg += rho0 dF (FP64), dF = 0
template <class R>
__global__ void k_fold(R* __restrict__ dF, double* __restrict__ dLdg, double rho0, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        dLdg[i] += rho0 * double(dF[i]);
        dF[i] = R(0);
    }
}

}  // namespace lbm
