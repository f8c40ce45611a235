"""Pins of the oracle's random draws and initial layout (Algorithm 3's random
start): the SplitMix64 output function against the published sequence of
the reference generator seeded with 0, the counter-based keying built on it,
the side of the initial box, and the initial coordinates as draws scaled to
that box; and the composition of layout steps into a level's layout."""
import numpy as np
import pytest

import workloads as W

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def _mix(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_splitmix64_published_sequence(oracle_mod):
    """The reference SplitMix64 generator (Steele, Lea, Flood 2014) seeded with
    0 returns 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f: the
    output function of its states G, 2G, 3G.  The oracle's keyed draw
    rand(seed, a, b) applies that function twice: to the state a + 1 steps
    from the seed, then, advanced b + 1 steps, to the result."""
    O = oracle_mod
    assert [_mix((k * GOLDEN) & M64) for k in (1, 2, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                          0x06C45D188009454F]
    rng = np.random.default_rng(3)
    for _ in range(200):
        seed, a, b = (int(v) for v in rng.integers(0, 2 ** 63, size=3, dtype=np.int64))
        a, b = a % (1 << 40), b % 1024
        want = _mix((_mix((seed + GOLDEN * (a + 1)) & M64) + GOLDEN * (b + 1)) & M64)
        assert O.rand64(seed, a, b) == want
    # the generators of the synthetic inputs use the same output function
    assert int(W.rand_u64(0, 0, 1)[0]) == _mix((_mix(GOLDEN) + GOLDEN) & M64)


@pytest.mark.parametrize("k,d", [(1, 2), (2, 2), (4096, 2), (4097, 2), (1000, 3), (1001, 3), (262144, 3),
                                 (81, 4), (82, 4)])
def test_initial_box_side(oracle_mod, k, d):
    """The random start of Algorithm 3 fills a box of unit point density: the
    smallest integer side s with s^d >= k."""
    s = oracle_mod.init_side(k, d)
    assert s ** d >= k and (s - 1) ** d < k


def test_initial_coordinates(oracle_mod):
    """Coordinate m of vertex v is the top 24 bits of its keyed draw as a
    fraction of 1, times the box side; unused coordinates are 0; the points
    fill the box evenly."""
    O = oracle_mod
    k, d, seed = 5000, 3, 11
    x = O.init_coords(k, d, seed)
    s = O.init_side(k, d)
    assert (x[:, d:] == 0).all() and (x[:, :d] >= 0).all() and (x[:, :d] < s).all()
    tag = 0x636f6f7264000000
    for v in (0, 1, 77, 4999):
        for m in range(d):
            r = O.rand64(seed ^ tag, v, m)
            assert x[v, m] == np.float32(np.float32((r >> 40) * 2.0 ** -24) * np.float32(s))
    hist = np.histogram(x[:, 0], bins=s, range=(0, s))[0]
    assert hist.min() > 0.5 * k / s and hist.max() < 1.5 * k / s


def test_level_layout_is_its_steps(oracle_mod):
    """A level's layout (Algorithm 4 for T steps) is T single steps with step
    lengths s0, 0.9 s0, 0.81 s0, ... from the level's initial step length, and
    it lowers the energy of the random start."""
    O = oracle_mod
    A = W.grid_laplacian_2d(24)
    hg = O.build_from_matrix("symmetric", A)
    x0 = O.init_coords(hg.k, 2, 5).astype(np.float64)
    T = 6
    xl = O.layout(hg, 2, x0, iters=T)
    x = x0.copy()
    s = O.step0(hg.k, 2, x0)
    for _ in range(T):
        x, _, _, _ = O.layout_step(hg, 2, x, s)
        s *= 0.9
    assert np.array_equal(xl, x)
    assert O.energy(hg, 2, xl) < O.energy(hg, 2, x0)


def test_parts_from_tree_covers_every_vertex_once(oracle_mod):
    """The owner map used by the cut checks: every vertex has exactly one
    owner, a leaf's vertices its range, a split node's its separator range."""
    O = oracle_mod
    A = W.powerlaw_symmetric(900, seed=2)
    hg = O.build_from_matrix("symmetric", A)
    for sbd in (False, True):
        perm, tree = O.order(hg, 3, O.init_coords(hg.k, 3, 2), seed=2, min_part=8, sbd=sbd)
        part = O.parts_from_tree(hg.k, perm, tree, sbd=sbd)
        assert (part >= 0).all()
        counts = np.bincount(part, minlength=len(tree["heap"]))
        for i in range(len(tree["heap"])):
            n1, n2, ns = (int(tree[f][i]) for f in ("n1", "n2", "nsep"))
            assert counts[i] == (n1 if n2 == 0 and ns == 0 else ns)
