"""Pins of the synthetic problem generators (closed forms, structure)."""
import math

import numpy as np

import workloads as w


def test_helmholtz_structure_and_symmetry():
    p = w.helmholtz7(6, 8)
    A = p.to_scipy()
    assert p.n == 216
    assert abs(A - A.T).max() == 0          # complex symmetric, not Hermitian
    nnz_row = np.diff(p.rowptr)
    assert nnz_row.max() == 7 and nnz_row.min() == 4
    h = 1 / 7
    assert np.isclose(A[0, 1], -1 / h ** 2)


def test_helmholtz_sine_modes_closed_form():
    # -Lap_h of sin(pi a x) sin(pi b y) sin(pi c z) on the interior grid is
    # (4/h^2) sum sin^2(pi a h / 2) times the mode (Dirichlet eigenvectors).
    n = 7
    p = w.helmholtz7(n, 8)
    h = p.params["h"]
    kappa2 = p.params["k"] ** 2 * (1 + 0.01j)
    A = p.to_scipy()
    g = np.arange(1, n + 1) * h
    for a, b, c in [(1, 1, 1), (2, 5, 3), (7, 1, 4)]:
        v = np.einsum("i,j,k->kji", np.sin(math.pi * a * g), np.sin(math.pi * b * g), np.sin(math.pi * c * g)).ravel()
        lam = 4 / h ** 2 * sum(math.sin(math.pi * t * h / 2) ** 2 for t in (a, b, c)) - kappa2
        assert np.allclose(A @ v, lam * v, rtol=1e-12, atol=1e-9)


def _gradient(prob):
    """Node -> edge difference on interior nodes (nodes at even doubled coordinates)."""
    nc = prob.params["nc"]
    coords = prob.coords
    nodes = {}
    for k in range(1, nc):
        for j in range(1, nc):
            for i in range(1, nc):
                nodes[(2 * i, 2 * j, 2 * k)] = len(nodes)
    G = np.zeros((prob.n, len(nodes)))
    for e, (X, Y, Z) in enumerate(coords):
        c = [X, Y, Z]
        ax = [t % 2 for t in c].index(1)
        lo = list(c); lo[ax] -= 1
        hi = list(c); hi[ax] += 1
        if tuple(hi) in nodes:
            G[e, nodes[tuple(hi)]] += 1
        if tuple(lo) in nodes:
            G[e, nodes[tuple(lo)]] -= 1
    return G


def test_yee_count_and_curl_of_gradient():
    p = w.yee_maxwell(5, 10)
    assert p.n == 3 * 5 * 4 ** 2
    A = p.to_scipy()
    assert abs(A - A.T).max() == 0
    assert np.diff(p.rowptr).max() <= 13
    # curl(grad phi) = 0 exactly, so A (G phi) = -kappa^2 G phi
    G = _gradient(p)
    phi = np.random.default_rng(0).standard_normal(G.shape[1])
    v = G @ phi
    kappa2 = p.params["k"] ** 2 * (1 + 0.01j)
    assert np.allclose(A @ v, -kappa2 * v, rtol=1e-12, atol=1e-6)


def test_counter_normal_reproducible_and_normal():
    rows = np.arange(200000, dtype=np.int64)
    z1 = w.counter_normal_complex(17, rows, 3)
    z2 = w.counter_normal_complex(17, rows, 3)
    assert np.array_equal(z1, z2)
    assert abs(np.mean(np.abs(z1) ** 2) - 1.0) < 0.02
    assert abs(np.mean(z1)) < 0.01
    # splitmix64 published first outputs for seed 0 (state increments by the golden gamma)
    first = w.splitmix64(np.array([0], dtype=np.uint64))[0]
    assert int(first) == 0xE220A8397B1DCDAF


def test_butterfly_bench_sizes():
    m = w.butterfly_bench_sizes()
    assert len(m) == 200 and m.min() >= 16 and m.max() <= 128
