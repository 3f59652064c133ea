"""Pins of the oracle's symmetric-tensor mode (Sec. 2.3: a symmetric positive-definite tensor at the
grid nodes, applied to the curl through the node assembly S_t = D^{-1/2} (1/8 sum R^T eps^-1 R)
D^{-1/2}, and the admission rule inside absorbing faces).  Each pin comes from outside the oracle's
own stencil code:
  * discrete dispersion: in a uniform rotated medium an eigenvector of the Fourier symbol
    S_t(k) (|s|^2 I - s s^T), s = 2 sin(k/2), evolves by the leapfrog recurrence of its eigenvalue;
  * reduction: an isotropic or diagonal node tensor is the diagonal update whose edge eps^-1 is the
    mean of the edge's end nodes (the one node of an edge at a non-periodic high face);
  * the assembly is symmetric with ||S_t|| <= 1 when every eigenvalue of eps is at least one (the
    reason the paper gives for keeping the vacuum time step);
  * the transposed steps satisfy the dot-product identity; the node-tensor cotangent matches
    central differences (diagonal and off-diagonal components);
  * the admission rule on its stated cases.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, gradient_replay, tensor_rejected
from paper_2609_30039_gb300 import workloads as W
from tests.oracle_adapter import oracle_from_scene, pec_mask_E

S = W.COURANT


def _uniform(shape, eps):
    nx, ny, nz = shape
    t = W.inv_tensor6(eps)
    return np.broadcast_to(t[:, None, None, None], (6, nz, ny, nx)).copy()


def _edge_positions(shape, a):
    nx, ny, nz = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = [i.astype(float), j.astype(float), k.astype(float)]
    r[a] = r[a] + 0.5
    return r


def _leapfrog(mu, n):
    """a_0 = a_1 = 1, a_{m+1} = (2 - S^2 mu) a_m - a_{m-1}: E^n of a mode started with H = 0."""
    a0, a1 = 1.0, 1.0
    if n == 0:
        return a0
    for _ in range(n - 1):
        a0, a1 = a1, (2.0 - S * S * mu) * a1 - a0
    return a1


@pytest.mark.parametrize("pqr", [(1, 1, 2), (2, 0, 1), (0, 0, 3)])
def test_eigenmodes_of_a_rotated_medium_follow_the_discrete_dispersion(pqr):
    shape = (8, 6, 10)
    eps = W.principal_eps((2.0, 3.0, 4.5), W.rotation(2, 0.4) @ W.rotation(0, 0.7))
    T = np.linalg.inv(eps)
    kvec = np.array([2 * math.pi * pqr[q] / shape[q] for q in range(3)])
    c = np.cos(kvec / 2.0)
    s = 2.0 * np.sin(kvec / 2.0)
    # symbol of S_t at k (phases at the edges' own positions): off-diagonal couplings average four
    # edges around each of two nodes, which gives the cos(k/2) factors
    St = T * np.outer(c, c)
    np.fill_diagonal(St, np.diag(T))
    P = np.dot(s, s) * np.eye(3) - np.outer(s, s)
    # M = St P is similar to the symmetric St^1/2 P St^1/2: real eigenvalues mu, eigenvectors St^1/2 w
    lam, U = np.linalg.eigh(St)
    half = U @ np.diag(np.sqrt(lam)) @ U.T
    mu, Wv = np.linalg.eigh(half @ P @ half)
    n_steps = 240
    for m in range(3):
        v = half @ Wv[:, m]
        assert np.allclose(St @ P @ v, mu[m] * v, atol=1e-12)
        v /= np.abs(v).max()
        o = Oracle(shape, S, periodic=(1, 1, 1))
        o.set_tensor(_uniform(shape, eps))
        for a in range(3):
            r = _edge_positions(shape, a)
            o.field(a)[...] = v[a] * np.cos(kvec[0] * r[0] + kvec[1] * r[1] + kvec[2] * r[2])
        e0 = [o.field(a).copy() for a in range(3)]
        o.step(n_steps)
        amp = _leapfrog(float(mu[m]), n_steps)
        err = max(np.abs(o.field(a) - amp * e0[a]).max() for a in range(3))
        assert err < 1e-10, (m, float(mu[m]), err)


def _edge_mean(t, a, periodic):
    """eps^-1 on the a-edges: the mean of the two end nodes, or the one node of an edge at the
    high face of a non-periodic axis."""
    ax = 2 - a
    m = 0.5 * (t + np.roll(t, -1, axis=ax))
    if not periodic[a]:
        sl = [slice(None)] * 3
        sl[ax] = -1
        m[tuple(sl)] = t[tuple(sl)]
    return m


@pytest.mark.parametrize("isotropic", [True, False])
def test_diagonal_node_tensors_reduce_to_the_diagonal_update_with_edge_means(isotropic):
    shape = (11, 9, 14)
    periodic = (0, 1, 0)
    sc = W.Scene(shape=shape, n_steps=60, cpml=(3, 0, 0, 0, 4, 3), kappa_max=3.0, alpha_max=0.05,
                 periodic=periodic)
    rng = np.random.default_rng(4)
    nx, ny, nz = shape
    t = np.zeros((6, nz, ny, nx))
    t[0] = 1.0 / rng.uniform(1.0, 6.0, (nz, ny, nx))
    t[1] = t[0] if isotropic else 1.0 / rng.uniform(1.0, 6.0, (nz, ny, nx))
    t[2] = t[0] if isotropic else 1.0 / rng.uniform(1.0, 6.0, (nz, ny, nx))
    wave = W.gaussian_pulse(60, 8.0, periods=1, delay=3)
    sc.sources = [W.Source(W.EY, (5, 0, 6), (6, ny, 7), wave), W.Source(W.EZ, (nx - 1, 2, nz - 2), (nx, 3, nz - 1), wave)]
    sc.monitors = [W.Monitor((1, 0, 8), (nx, ny, 9), (0, 1, 2, 3, 4, 5), W.omegas_for((7.0, 9.0)))]
    ref = W.Scene(**{**sc.__dict__, "inv_eps": [_edge_mean(t[a], a, periodic) for a in range(3)]})
    sc.tensor = t
    o_t = oracle_from_scene(sc)
    o_d = oracle_from_scene(ref)
    D = [o_t.tensor_D(a) for a in range(3)]
    pec = pec_mask_E(shape, periodic)
    for a in range(3):
        # D counts the end nodes an edge has (1/2 each): 1, or 1/2 at a non-periodic high face
        want = np.ones((nz, ny, nx))
        if not periodic[a]:
            sl = [slice(None)] * 3
            sl[2 - a] = -1
            want[tuple(sl)] = 0.5
        assert np.array_equal(D[a][~pec[a]], want[~pec[a]])
    o_t.step(sc.n_steps)
    o_d.step(sc.n_steps)
    for c in range(6):
        ref_f = o_d.field(c)
        assert np.abs(o_t.field(c) - ref_f).max() <= 1e-12 * np.abs(ref_f).max(), c
    F_t, F_d = o_t.dft(0), o_d.dft(0)
    assert np.linalg.norm(F_t - F_d) <= 1e-12 * np.linalg.norm(F_d)


def _random_admitted_tensors(rng, shape, lo=1.0, hi=5.0):
    """Random SPD eps per node with eigenvalues in [lo, hi] and random principal axes."""
    nx, ny, nz = shape
    n = nx * ny * nz
    Q, _ = np.linalg.qr(rng.standard_normal((n, 3, 3)))
    lam = rng.uniform(lo, hi, (n, 3))
    eps = np.einsum("nij,nj,nkj->nik", Q, lam, Q)
    return W.inv_tensor6(eps).reshape(6, nz, ny, nx)


def test_assembly_is_symmetric_and_bounded_by_one_when_eps_is_at_least_one():
    shape = (5, 6, 7)
    rng = np.random.default_rng(9)
    o = Oracle(shape, S, periodic=(0, 1, 0))
    o.set_tensor(_random_admitted_tensors(rng, shape))
    pec = pec_mask_E(shape, (0, 1, 0))
    nz, ny, nx = shape[::-1]

    def rnd():
        v = [rng.standard_normal((nz, ny, nx)) for _ in range(3)]
        for a in range(3):
            v[a][pec[a]] = 0.0
        return v

    def dot(u, v):
        return sum(float((x * y).sum()) for x, y in zip(u, v))

    u, v = rnd(), rnd()
    Su, Sv = o.tensor_apply(u), o.tensor_apply(v)
    assert abs(dot(u, Sv) - dot(Su, v)) <= 1e-14 * math.sqrt(dot(u, u) * dot(v, v))
    # the largest eigenvalue by power iteration (S_t is symmetric positive semidefinite)
    x = rnd()
    for _ in range(300):
        y = o.tensor_apply(x)
        nrm = math.sqrt(dot(y, y))
        x = [a / nrm for a in y]
    lam = dot(x, o.tensor_apply(x))
    assert 0.5 < lam <= 1.0 + 1e-12, lam
    # a vacuum node tensor gives the identity on every unknown edge
    o.set_tensor(_uniform(shape, np.eye(3)))
    w = o.tensor_apply(u)
    for a in range(3):
        assert np.allclose(w[a], u[a], rtol=1e-15, atol=0.0)


def _tensor_scene(shape=(10, 9, 16), steps=40, design=None):
    """CPML on the z faces holding diagonal tensors whose normal (z) eigenvalue is not
    intermediate, rotated tensors inside, PEC x and y faces."""
    rng = np.random.default_rng(21)
    nx, ny, nz = shape
    sc = W.Scene(shape=shape, n_steps=steps, cpml=(0, 0, 0, 0, 4, 4), kappa_max=3.0, alpha_max=0.05)
    t = _random_admitted_tensors(rng, shape, 1.0, 4.0)
    d = np.zeros_like(t)
    d[0], d[1] = 1.0 / 2.0, 1.0 / 3.0
    d[2] = 1.0 / 1.5   # eps_zz = 1.5 below both tangential eigenvalues
    t[:, :4], t[:, nz - 4:] = d[:, :4], d[:, nz - 4:]
    sc.tensor = t
    wave = W.gaussian_pulse(steps, 7.0, periods=1, delay=3)
    sc.sources = [W.Source(W.EX, (3, 3, 6), (7, 6, 7), wave)]
    sc.monitors = [W.Monitor((1, 1, nz - 6), (nx, ny, nz - 5), (0, 1, 3, 4), W.omegas_for((6.0, 8.0)))]
    sc.design = design
    return sc


@pytest.mark.parametrize("nsteps", [1, 7])
def test_transposed_tensor_steps_satisfy_the_dot_product_identity(nsteps):
    sc = _tensor_scene()
    assert not tensor_rejected(sc.tensor, sc.shape, sc.cpml).any()
    o = oracle_from_scene(sc, with_sources=False, with_monitors=False)
    rng = np.random.default_rng(30 + nsteps)
    pec = pec_mask_E(sc.shape)

    def rnd():
        x = rng.standard_normal(o.state_len)
        for a in range(3):
            x[a * o.n:(a + 1) * o.n].reshape(sc.shape[::-1])[pec[a]] = 0.0
        return x

    x, y = rnd(), rnd()
    o.set_state(x, step=0)
    o.step(nsteps)
    fx = o.get_state()
    o.adj_reset()
    o.set_state(y, adjoint=True)
    for m in reversed(range(nsteps)):
        o.adjoint_step(m)
    fty = o.get_state(adjoint=True)
    lhs, rhs = float(fx @ y), float(x @ fty)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(fx) * np.linalg.norm(y), (lhs, rhs)


def _objective(o):
    F = o.dft(0)
    return float((np.abs(F) ** 2).sum()), {0: 2.0 * F}


def test_node_tensor_cotangent_matches_central_differences():
    box = ((3, 2, 6), (7, 6, 10))
    sc = _tensor_scene(design=box)
    o = oracle_from_scene(sc)
    J0 = gradient_replay(o, sc.n_steps, _objective)
    g = np.stack([o.grad(q) for q in range(6)])
    (lx, ly, lz), (hx, hy, hz) = box
    rng = np.random.default_rng(8)
    d = rng.standard_normal(g.shape)
    base = sc.tensor.copy()

    def J_h(h, comps=range(6)):
        t = base.copy()
        for q in comps:
            t[q, lz:hz, ly:hy, lx:hx] += h * d[q]
        sc2 = W.Scene(**{**sc.__dict__, "tensor": t, "design": None})
        o2 = oracle_from_scene(sc2)
        o2.step(sc.n_steps)
        return _objective(o2)[0]

    h = 1e-6
    for comps in ((0, 1, 2), (3, 4, 5)):
        dirderiv = float(sum((g[q] * d[q]).sum() for q in comps))
        fd = (J_h(h, comps) - J_h(-h, comps)) / (2 * h)
        assert abs(fd - dirderiv) <= 1e-6 * abs(dirderiv), (comps, fd, dirderiv)
    dirderiv = float((g * d).sum())
    r1 = abs(J_h(1e-3) - J0 - 1e-3 * dirderiv)
    r2 = abs(J_h(5e-4) - J0 - 5e-4 * dirderiv)
    assert 3.6 < r1 / r2 < 4.4, (r1, r2)


def test_admission_rule_cases():
    shape = (4, 4, 12)
    nx, ny, nz = shape
    cpml = (0, 0, 0, 0, 3, 3)

    def one(eps, k):
        t = _uniform(shape, np.eye(3))
        t[:, k, 1, 2] = W.inv_tensor6(eps)
        return tensor_rejected(t, shape, cpml)[k, 1, 2]

    R = W.rotation(0, 0.3)
    uni_normal_low = W.principal_eps((3.0, 3.0, 1.5))
    assert not one(np.eye(3), 0)
    assert not one(uni_normal_low, 1)                             # normal eigenvalue the smallest
    assert not one(W.principal_eps((2.0, 3.0, 4.0)), 0)           # the largest
    assert one(W.principal_eps((2.0, 4.0, 3.0)), 0)               # intermediate normal eigenvalue
    assert not one(W.principal_eps((2.0, 4.0, 3.0)), 6)           # the same outside the slabs
    assert one(W.principal_eps((2.0, 3.0, 4.0), R), 11)           # z is not a principal axis
    assert not one(W.principal_eps((2.0, 3.0, 4.0), R), 5)        # allowed away from the faces
    assert not one(W.principal_eps((2.0, 3.0, 4.0), W.rotation(2, 0.8)), 2)   # rotated about the normal
    assert one(W.principal_eps((0.8, 3.0, 4.0)), 6)               # eps below one
    assert one(-np.eye(3), 6)                                     # not positive definite
    # equal normal and tangential eigenvalues are not intermediate
    assert not one(W.principal_eps((2.0, 3.0, 3.0)), 0)


@pytest.mark.parametrize("eps,rejected", [
    (W.principal_eps((2.0, 3.0, 1.5)), False),                       # normal eigenvalue the smallest
    (W.principal_eps((2.0, 3.0, 4.0), W.rotation(2, 0.6)), False),   # rotated about the normal
    (W.principal_eps((1.5, 4.0, 8.0), W.rotation(0, 0.6)), True),    # normal not a principal axis
    (W.principal_eps((1.5, 8.0, 4.0)), True),                        # intermediate normal eigenvalue
])
def test_rejected_tensors_grow_inside_absorbing_faces_and_admitted_ones_do_not(eps, rejected):
    # the long-time behaviour behind the admission rule (Sec. 2.3, App. A): a uniform tensor fills a
    # domain whose z faces absorb; over the last 1000 of 4000 steps from random fields a rejected
    # tensor grows exponentially, an admitted one at most linearly (the zero-frequency part of the
    # random start)
    shape = (6, 6, 40)
    cpml = (0, 0, 0, 0, 8, 8)
    t = _uniform(shape, eps)
    assert bool(tensor_rejected(t, shape, cpml).any()) == rejected
    o = Oracle(shape, S, periodic=(1, 1, 0), cpml=cpml, alpha_max=0.05)
    o.set_tensor(t)
    x = np.zeros(o.state_len)
    x[:6 * o.n] = np.random.default_rng(0).standard_normal(6 * o.n)
    o.set_state(x, step=0)
    o.step(3000)
    n3 = np.linalg.norm(o.get_state()[:6 * o.n])
    o.step(1000)
    r = np.linalg.norm(o.get_state()[:6 * o.n]) / n3
    assert (r > 10.0) if rejected else (r < 2.0), r
