"""The closed form the 3-D kernel's collision relies on, checked against the
oracle's literal matrices.

Both 3-D scalar lattices relax every central moment except the three
first-order ones to its Maxwellian equilibrium, s mu(m) mu(n) mu(p) with
mu = (1, 0, cs^2).  The post-collision central moments are then
    s (mu x mu x mu) + k'_x [100] + k'_y [010] + k'_z [001],
and because P and F(u) are Kronecker products of their one-dimensional
factors, the outgoing populations factor per axis:
    s A_x A_y A_z + k'_x B_x C_y C_z + k'_y C_x B_y C_z + k'_z C_x C_y B_z,
with A, B, C the 1-D factors P1^-1 F1^-1(u) applied to (1, 0, cs^2),
(0, 1, 0) and (1, 0, 0).  This test builds the post-collision populations
both ways for random states -- the literal way with the oracle's 27 x 27
P^-1 and F^-1(u), the factorised way from the closed-form 1-D factors -- and
requires agreement to rounding.  It also checks that the collision of the
literal matrices (relax k with w, everything else to equilibrium) uses only
the zeroth and first raw moments of the incoming populations.
"""
import numpy as np

import oracle

CS2 = 1.0 / 3.0


def one_d_factors(u):
    """A, B, C over e = (0, +1, -1): P1^-1 F1^-1(u) of the three 1-D central
    moment vectors, written out from raw moments (1, u, cs2 + u^2),
    (0, 1, 2u) and (1, u, u^2) and p(0) = M0 - M2, p(+-1) = (M2 +- M1) / 2."""
    t = CS2 + u * u
    A = np.array([1 - t, 0.5 * (t + u), 0.5 * (t - u)])
    B = np.array([-2 * u, u + 0.5, u - 0.5])
    C = np.array([1 - u * u, 0.5 * (u * u + u), 0.5 * (u * u - u)])
    return A, B, C


def factorised(s, k, u):
    (Ax, Bx, Cx), (Ay, By, Cy), (Az, Bz, Cz) = [one_d_factors(v) for v in u]
    out = np.empty(27)
    for c in range(3):
        for b in range(3):
            for a in range(3):
                out[a + 3 * b + 9 * c] = (s * Ax[a] * Ay[b] * Az[c] + k[0] * Bx[a] * Cy[b] * Cz[c]
                                          + k[1] * Cx[a] * By[b] * Cz[c] + k[2] * Cx[a] * Cy[b] * Bz[c])
    return out


def library_order_to_oracle():
    """Index map from the kernel's velocity order (a + 3b + 9c over
    e = 0, +1, -1 per axis) to the oracle's."""
    E = [0, 1, -1]
    idx = {tuple(v): i for i, v in enumerate(oracle.velocities3())}
    return np.array([idx[(E[q % 3], E[(q // 3) % 3], E[q // 9])] for q in range(27)])


def moment_index(m, n, p):
    return m + 3 * n + 9 * p   # the oracle's moment order (k % 3, (k / 3) % 3, k / 9)


def test_factorised_outputs_equal_the_matrix_form():
    rng = np.random.default_rng(11)
    perm = library_order_to_oracle()
    Pinv = oracle.matrix3("Pinv")
    for _ in range(50):
        u = rng.uniform(-0.2, 0.2, 3)
        s = rng.uniform(-0.5, 1.5)
        k = rng.uniform(-0.05, 0.05, 3)
        cm = np.zeros(27)
        mu = (1.0, 0.0, CS2)
        for p in range(3):
            for n in range(3):
                for m in range(3):
                    cm[moment_index(m, n, p)] = s * mu[m] * mu[n] * mu[p]
        cm[moment_index(1, 0, 0)], cm[moment_index(0, 1, 0)], cm[moment_index(0, 0, 1)] = k
        literal = Pinv @ (oracle.matrix3("Finv", *u) @ cm)
        got = factorised(s, k, u)
        assert np.abs(got - literal[perm]).max() < 1e-14


def test_collision_depends_only_on_zeroth_and_first_moments():
    """Two incoming population sets with equal s and j (different higher
    moments) leave the same post-collision populations."""
    rng = np.random.default_rng(12)
    P = oracle.matrix3("P")
    Pinv = oracle.matrix3("Pinv")
    for _ in range(20):
        u = rng.uniform(-0.2, 0.2, 3)
        F = oracle.matrix3("F", *u)
        Fi = oracle.matrix3("Finv", *u)
        w = rng.uniform(0.5, 1.9)
        q = rng.uniform(-0.03, 0.03, 3)
        a = rng.uniform(0.0, 0.1, 27)
        # change every raw moment of order >= 2, keep order 0 and 1
        raw = P @ a
        for kk in range(27):
            if (kk % 3) + ((kk // 3) % 3) + kk // 9 >= 2:
                raw[kk] += rng.uniform(-0.02, 0.02)
        b = Pinv @ raw

        def collide(pops):
            cm = F @ (P @ pops)
            s0 = cm[0]
            eq = np.array([s0 * (1.0, 0.0, CS2)[kk % 3] * (1.0, 0.0, CS2)[(kk // 3) % 3]
                           * (1.0, 0.0, CS2)[kk // 9] for kk in range(27)])
            for i, kk in enumerate((1, 3, 9)):
                eq[kk] = q[i]
            lam = np.array([w if (kk % 3) + ((kk // 3) % 3) + kk // 9 == 1 else 1.0 for kk in range(27)])
            return Pinv @ (Fi @ (cm + lam * (eq - cm)))

        assert np.abs(collide(a) - collide(b)).max() < 1e-14
