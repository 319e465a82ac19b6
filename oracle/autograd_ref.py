"""FP64 CPU reference gradient of a flow functional with respect to a body-force field.

TEST INFRASTRUCTURE ONLY (used by the tests to check the library's adjoint).  This is a
vectorised restatement, in plain torch float64 CPU operations, of the oracle's D3Q19 MRT step
(periodic box, Guo-type force field, Smagorinsky closure by 6 fixed-point sweeps, Yu's strain
rate, eq. (LuoS)); torch.autograd differentiates it.  The tests first check that its forward
pass equals the C oracle (lbm_oracle.c) to rounding, so the gradient is that of the oracle's map.

Functional (total dissipation at the final time): L = sum_x nu_eff(x) sum_ab S_ab(x)^2, with
nu_eff = (tau - 1/2)/3 and S, tau of the pre-collision state that step T+1 would see.
"""
import numpy as np
import torch

from . import tables

CS2 = 1.0 / 3.0


class Model:
    def __init__(self, rates, smag_cs, smag_iters=6, rho0=1.0):
        c, w, T, Ti, opp = tables(19)
        self.c = torch.tensor(c, dtype=torch.float64)
        self.ci = c
        self.w = torch.tensor(w, dtype=torch.float64)
        self.T = torch.tensor(T, dtype=torch.float64)
        self.Ti = torch.tensor(Ti, dtype=torch.float64)
        self.s = torch.tensor(rates, dtype=torch.float64)
        self.nu_idx = [9, 11, 13, 14, 15]
        self.tau0 = 1.0 / rates[9]
        self.cs = smag_cs
        self.K = smag_iters
        self.rho0 = rho0

    # pull streaming on a periodic box: p_i(x) = f_i(x - c_i); arrays (19, nz, ny, nx)
    def pull(self, f):
        return torch.stack([torch.roll(f[i], shifts=(int(self.ci[i, 2]), int(self.ci[i, 1]), int(self.ci[i, 0])),
                                       dims=(0, 1, 2)) for i in range(19)])

    def meq(self, drho, j):
        """eq. (meq), moment order of eq. (moment), w_eps = 3, w_epsj = -11/2, w_xx = -1/2."""
        r0 = self.rho0
        jx, jy, jz = j[0], j[1], j[2]
        jj = jx * jx + jy * jy + jz * jz
        z = torch.zeros_like(drho)
        m9 = (3 * jx * jx - jj) / r0
        m11 = (jy * jy - jz * jz) / r0
        return torch.stack([drho, -11 * drho + 19 * jj / r0, 3 * drho - 5.5 * jj / r0, jx, -2 * jx / 3, jy, -2 * jy / 3,
                            jz, -2 * jz / 3, m9, -0.5 * m9, m11, -0.5 * m11, jx * jy / r0, jy * jz / r0, jx * jz / r0,
                            z, z, z])

    def fbar(self, j, F):
        """Guo-type discrete force per population."""
        u = j / self.rho0
        cu = torch.einsum("ia,a...->i...", self.c, u)
        cF = torch.einsum("ia,a...->i...", self.c, F)
        uF = (u * F).sum(0)
        return self.w.view(19, *([1] * u[0].dim())) * ((cF - uF) / CS2 + cu * cF / (CS2 * CS2))

    def strain_yu(self, mn, s1, snu):
        r0 = self.rho0
        m1, m9, m11 = mn[1], mn[9], mn[11]
        return torch.stack([-(s1 * m1 + 19 * snu * m9) / (38 * r0),
                            -(2 * s1 * m1 - 19 * snu * (m9 - 3 * m11)) / (76 * r0),
                            -(2 * s1 * m1 - 19 * snu * (m9 + 3 * m11)) / (76 * r0),
                            -3 * snu * mn[13] / (2 * r0), -3 * snu * mn[14] / (2 * r0), -3 * snu * mn[15] / (2 * r0)])

    @staticmethod
    def snorm(S):
        ss = S[0] ** 2 + S[1] ** 2 + S[2] ** 2 + 2 * (S[3] ** 2 + S[4] ** 2 + S[5] ** 2)
        return torch.sqrt(2 * ss)

    def state(self, p, F):
        """Moments, closure and strain rate of pulled populations p under force F."""
        m = torch.einsum("ki,i...->k...", self.T, p)
        drho = m[0]
        j = torch.stack([m[3], m[5], m[7]]) + 0.5 * F
        meq = self.meq(drho, j)
        TF = torch.einsum("ki,i...->k...", self.T, self.fbar(j, F))
        mn = m - meq + 0.5 * TF
        tau = torch.full_like(drho, self.tau0)
        for _ in range(self.K):
            S = self.strain_yu(mn, self.s[1], 1.0 / tau)
            tau = self.tau0 + 3 * self.cs * self.cs * self.snorm(S)
        S = self.strain_yu(mn, self.s[1], 1.0 / tau)
        return m, meq, TF, tau, S

    def collide(self, p, F):
        m, meq, TF, tau, S = self.state(p, F)
        shape = (19,) + (1,) * (m.dim() - 1)
        svec = self.s.view(shape).expand_as(m).clone()
        for k in self.nu_idx:
            svec[k] = 1.0 / tau
        mstar = m - svec * (m - meq) + (1 - 0.5 * svec) * TF
        return torch.einsum("ik,k...->i...", self.Ti, mstar)

    def step(self, f, F):
        return self.collide(self.pull(f), F)

    def loss(self, f, F):
        _, _, _, tau, S = self.state(self.pull(f), F)
        nu = (tau - 0.5) / 3
        SS = S[0] ** 2 + S[1] ** 2 + S[2] ** 2 + 2 * (S[3] ** 2 + S[4] ** 2 + S[5] ** 2)
        return (nu * SS).sum()


def loss_and_grad(f0, g, rates, smag_cs, steps, rho0=1.0, segment=None):
    """L(g) after `steps` steps from the post-collision state f0 (19, nz, ny, nx) under the force
    density rho0 g (3, nz, ny, nx), and dL/dg.  segment: recompute in segments of that many steps
    (torch checkpointing) to bound memory."""
    M = Model(rates, smag_cs, rho0=rho0)
    gt = torch.tensor(np.asarray(g, dtype=np.float64), requires_grad=True)
    f = torch.tensor(np.asarray(f0, dtype=np.float64))
    F = rho0 * gt
    if segment:
        from torch.utils.checkpoint import checkpoint

        def seg(fin, Fin, n):
            for _ in range(n):
                fin = M.step(fin, Fin)
            return fin

        done = 0
        while done < steps:
            n = min(segment, steps - done)
            f = checkpoint(seg, f, F, n, use_reentrant=False)
            done += n
    else:
        for _ in range(steps):
            f = M.step(f, F)
    L = M.loss(f, F)
    L.backward()
    return float(L.detach()), gt.grad.numpy().copy(), f.detach().numpy()
