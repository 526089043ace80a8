"""Pins of the far-field oracle (Sec. "Far-field Computation") and of its Ewald
reference, against facts that do not come from the oracle itself: harmonicity
of 1/r, independence of the Ewald split, absolute convergence of high-order
image sums, closed forms near a particle, lattice symmetry, and the paper's
own Ewald-test error figures."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def _paper(name):
    for line in open(GOLDEN):
        if line.startswith(name + " "):
            return float(line.split()[1])
    raise KeyError(name)


def _where(p):
    return {t: q for q, t in enumerate(oracle.multipole_index(p))}


@pytest.mark.parametrize("K,box", [(6, 1.0), (7, 2.5)])
def test_derivatives_trace_is_background_density(K, box):
    # The periodic potential with a neutralising background obeys
    # lap Phi = 4 pi / V away from the lattice points, so every trace of the
    # derivatives tensor vanishes except the second-order one.
    p = 8
    D = oracle.derivatives(K, 2, p, box)
    wh = _where(p)
    V = box ** 3
    for (a, b, c) in oracle.multipole_index(p - 2):
        tr = D[:, wh[(a + 2, b, c)]] + D[:, wh[(a, b + 2, c)]] + D[:, wh[(a, b, c + 2)]]
        ref = 4 * np.pi / V if (a, b, c) == (0, 0, 0) else 0.0
        scale = np.abs(D[:, wh[(a + 2, b, c)]]).max()
        assert np.abs(tr - ref).max() <= 1e-11 * scale


def test_derivatives_do_not_depend_on_the_ewald_split():
    D1 = oracle.derivatives(8, 2, 8, alpha=3.5)
    D2 = oracle.derivatives(8, 2, 8, alpha=2.8, nimg=3, hmax=8)
    scale = np.abs(D1).max(axis=0)
    assert (np.abs(D1 - D2).max(axis=0) / scale).max() < 1e-11


def test_derivatives_parity_and_axis_symmetry():
    K, p = 7, 6
    D = oracle.derivatives(K, 2, p).reshape(K, K, K, -1)
    idx = oracle.multipole_index(p)
    wh = _where(p)
    neg = lambda i: (-i) % K
    g = np.arange(K)
    Dm = D[np.ix_(neg(g), neg(g), neg(g))]
    sign = np.array([(-1.0) ** sum(t) for t in idx])
    assert np.allclose(Dm, sign * D, rtol=0, atol=1e-12 * np.abs(D).max())
    # swapping the x and y axes of the grid swaps the a and b indices
    swap = np.array([wh[(b, a, c)] for (a, b, c) in idx])
    assert np.allclose(D.transpose(1, 0, 2, 3)[..., swap], D, rtol=0, atol=1e-12 * np.abs(D).max())


def test_high_orders_equal_the_direct_image_sum():
    # From order 6 on the image sum converges absolutely (terms ~ |n|^-7):
    # summing the derivatives of 1/r over a cube of images must give D.
    K, R, p, nmax = 6, 2, 8, 10
    D = oracle.derivatives(K, R, p)
    idx = oracle.multipole_index(p)
    high = np.array([sum(t) >= 6 for t in idx])
    w = 1.0 / K
    for g in [(3, 0, 0), (2, 5, 1), (0, 0, 0), (1, 1, 4)]:
        c = [x - K if 2 * x > K else x for x in g]
        near = all(abs(x) <= R for x in c)
        acc = np.zeros(len(idx))
        for nx in range(-nmax, nmax + 1):
            for ny in range(-nmax, nmax + 1):
                for nz in range(-nmax, nmax + 1):
                    if near and nx == ny == nz == 0:
                        continue
                    r = (c[0] * w + nx, c[1] * w + ny, c[2] * w + nz)
                    acc += oracle.coulomb_derivatives(p, r)
        row = D[(g[0] * K + g[1]) * K + g[2]]
        scale = np.abs(row[high]).max()
        assert np.abs(acc[high] - row[high]).max() < 2e-4 * scale


def test_fft_convolution_equals_the_direct_cyclic_sum():
    rng = np.random.default_rng(3)
    K, p = 5, 5
    D = oracle.derivatives(K, 2, p)
    M = rng.standard_normal((K ** 3, oracle.multipole_terms(p)))
    Td = oracle.convolve_direct(K, p, D, M)
    Tf = oracle.taylors_fft(K, p, D, M)
    assert np.abs(Td - Tf).max() < 1e-10 * np.abs(Td).max()


def test_taylor_forces_are_the_gradient_of_the_polynomial():
    p, K = 4, 3
    idx = oracle.multipole_index(p)
    T = np.zeros((K ** 3, len(idx)))
    T[:, idx.index((2, 1, 0))] = 1.0
    T[:, idx.index((0, 0, 3))] = -2.0
    pos = np.random.default_rng(1).random((64, 3)).astype(np.float32)
    a = oracle.taylor_forces(pos, 1.0, K, p, T)
    _, rel, perm = oracle.bin_particles(pos, 1.0, K)
    x = np.empty((64, 3))
    x[perm] = rel[:, :3].astype(np.float64) / K
    ref = np.stack([2 * x[:, 0] * x[:, 1], x[:, 0] ** 2, -6 * x[:, 2] ** 2], 1)
    assert np.abs(a - ref).max() < 1e-15


def test_ewald_pair_at_small_separation():
    # Phi(r) = 1/r + (2 pi / 3V) r^2 + const + O(r^4) near a particle of a cubic
    # lattice with a neutralising background (lap = 4 pi / V, cubic symmetry):
    # a = m (-r/r^3 + (4 pi / 3V) r) to O(r^5) relative.
    r = np.array([0.01, 0.004, -0.007])
    x0 = np.array([0.3, 0.6, 0.2])
    pos = np.array([x0 + r, x0], np.float32)
    rr = pos[0].astype(np.float64) - pos[1]
    a = oracle.ewald_forces(pos, 1.0)
    d = np.linalg.norm(rr)
    ref = 0.5 * (-rr / d ** 3 + 4 * np.pi / 3 * rr)
    assert np.linalg.norm(a[0] - ref) < 1e-8 * np.linalg.norm(ref)
    assert np.abs(a[0] + a[1]).max() < 1e-12 * np.linalg.norm(ref)


def test_ewald_split_independence_and_momentum():
    pos = np.random.default_rng(5).random((300, 3)).astype(np.float32)
    a1 = oracle.ewald_forces(pos, 1.0)
    a2 = oracle.ewald_forces(pos, 1.0, alpha=2.5, nimg=2, hmax=7)
    assert np.abs(a1 - a2).max() < 1e-11 * np.abs(a1).max()
    assert np.abs(a1.sum(axis=0)).max() < 1e-12 * np.abs(a1).max()


def test_lattice_forces_vanish():
    # one particle at every cell centre: every force is zero by symmetry
    K = 8
    g = (np.arange(K) + 0.5) / K
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    scale = (1.0 / K ** 3) * K ** 2           # m / w^2
    assert np.abs(oracle.far_field(pos, 1.0, K, 2, 8)).max() < 1e-12 * scale
    assert np.abs(oracle.ewald_forces(pos, 1.0, sinks=np.arange(0, K ** 3, 37))).max() < 1e-11 * scale


def test_single_particle_feels_no_force_from_its_images():
    pos = np.array([[0.37, 0.61, 0.12]], np.float32)
    assert np.abs(oracle.far_field(pos, 1.0, 6, 2, 8)).max() < 1e-13


def test_error_falls_with_multipole_order():
    rng = np.random.default_rng(7)
    N, K, R = 4096, 8, 2
    pos = rng.random((N, 3)).astype(np.float32)
    sinks = np.sort(rng.choice(N, 256, replace=False))
    ref = oracle.ewald_forces(pos, 1.0, sinks=sinks)
    near = oracle.forces(pos, 1.0, K, R, 1e-6, sinks=sinks)
    med = []
    for p in (4, 6, 8):
        far = oracle.far_field(pos, 1.0, K, R, p)[sinks]
        med.append(np.median(oracle.frac_error(near + far, ref)))
    assert med[0] > 3 * med[1] > 9 * med[2]
    assert med[2] < 5e-5


def test_paper_ewald_configuration():
    # The paper's Ewald test: 65536 random particles, CPD 11, multipole order 8;
    # its median and 99th-percentile fractional errors (1.1e-5..1.2e-5 and
    # 1.4e-4..1.6e-4) bound ours within a factor of two.
    N = int(_paper("ewald_test_particles"))
    K = int(_paper("ewald_test_cpd"))
    p = int(_paper("ewald_test_order"))
    rng = np.random.default_rng(11)
    pos = rng.random((N, 3)).astype(np.float32)
    pos[pos >= 1.0] = 0.0
    eps = 1e-5
    sinks = np.sort(rng.choice(N, 256, replace=False))
    # no pair closer than the softening length, so the near field is Newtonian
    from scipy.spatial import cKDTree
    assert not cKDTree(pos.astype(np.float64), boxsize=1.0).query_pairs(2.16 * eps)
    ref = oracle.ewald_forces(pos, 1.0, sinks=sinks)
    tot = oracle.forces(pos, 1.0, K, 2, eps, sinks=sinks) + oracle.far_field(pos, 1.0, K, 2, p)[sinks]
    fe = oracle.frac_error(tot, ref)
    med, p99 = np.median(fe), np.percentile(fe, 99)
    assert _paper("ewald_median_err") / 2 < med < 2 * 1.2e-5
    assert _paper("ewald_p99_err") / 2 < p99 < 2 * 1.6e-4


def _closed_form_coulomb(r, a, b, c):
    """d^a/dx^a d^b/dy^b d^c/dz^c of 1/|r| for a + b + c <= 3, from the
    textbook tensors: 1/r; -x_i/r^3; 3 x_i x_j/r^5 - delta_ij/r^3;
    -15 x_i x_j x_k/r^7 + 3 (delta_ij x_k + delta_ik x_j + delta_jk x_i)/r^5."""
    x = np.asarray(r, np.float64)
    d = float(np.linalg.norm(x))
    ax = [0] * a + [1] * b + [2] * c
    dl = lambda i, j: 1.0 if i == j else 0.0
    if len(ax) == 0:
        return 1.0 / d
    if len(ax) == 1:
        return -x[ax[0]] / d ** 3
    if len(ax) == 2:
        i, j = ax
        return 3 * x[i] * x[j] / d ** 5 - dl(i, j) / d ** 3
    i, j, k = ax
    return (-15 * x[i] * x[j] * x[k] / d ** 7
            + 3 * (dl(i, j) * x[k] + dl(i, k) * x[j] + dl(j, k) * x[i]) / d ** 5)


POINTS = [(0.7, -0.4, 0.3), (-1.3, 0.2, 2.1), (0.05, 0.9, -0.6)]


@pytest.mark.parametrize("r", POINTS)
def test_coulomb_derivatives_low_orders_equal_closed_forms(r):
    # Orders 0..3 of the derivatives of 1/r against the textbook tensors
    # (a route that shares nothing with the Hermite recursion).
    p = 3
    D = oracle.coulomb_derivatives(p, r)
    for q, (a, b, c) in enumerate(oracle.multipole_index(p)):
        ref = _closed_form_coulomb(r, a, b, c)
        assert abs(D[q] - ref) <= 1e-13 * max(1.0, abs(ref)) * np.linalg.norm(r) ** -(1 + a + b + c), \
            ((a, b, c), D[q], ref)


@pytest.mark.parametrize("r", POINTS)
def test_coulomb_derivatives_each_order_differentiates_the_one_below(r):
    # Orders 4..p: every term must be the derivative, along one of its axes, of
    # the term one order below, taken by fourth-order central differences of
    # the oracle's own lower-order values.  With orders <= 3 pinned to the
    # closed forms this pins every order of the recursion.
    p = 10
    h = 1e-3
    wh_lo = _where(p - 1)
    idx = oracle.multipole_index(p)
    D = oracle.coulomb_derivatives(p, r)
    x = np.asarray(r, np.float64)
    steps = {}
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        steps[ax] = [oracle.coulomb_derivatives(p - 1, x + s * e) for s in (2, 1, -1, -2)]
    d = float(np.linalg.norm(x))
    for q, t in enumerate(idx):
        m = sum(t)
        if m < 4:
            continue
        for ax in range(3):
            if t[ax] == 0:
                continue
            lo = list(t)
            lo[ax] -= 1
            f2, f1, m1, m2 = (v[wh_lo[tuple(lo)]] for v in steps[ax])
            fd = (-f2 + 8 * f1 - 8 * m1 + m2) / (12 * h)
            scale = d ** -(m + 1) * np.prod([float(k) for k in range(1, m + 1)])  # |D^m| <= m!/r^(m+1)
            assert abs(D[q] - fd) <= 2e-7 * scale, (t, ax, D[q], fd)
