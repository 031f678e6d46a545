"""The seeded synthetic inputs follow the recipe stated for each workload:
sizes, charge neutrality, wall margins, size distributions, arrival times,
and determinism in the seed."""
import numpy as np

from paper_1806_04801_gb300 import inputs as I


def test_small_and_large_periodic_workloads():
    xyz, q = I.small_periodic()
    assert xyz.shape == (1000, 3) and q.shape == (1000,)
    assert np.all((xyz >= 0) & (xyz < 1)) and q.sum() == 0 and set(np.unique(q)) == {-1.0, 1.0}
    xyz, q = I.large_periodic()
    assert xyz.shape == (100_000, 3) and np.all((xyz >= 0) & (xyz < 1))
    assert abs(q.sum()) <= 1e-12 * np.abs(q).sum()
    assert 0.95 < q.std() < 1.05  # N(0, 1) minus the mean


def test_grounded_cavity_keeps_off_the_walls():
    xyz, q = I.grounded_cavity()
    L = np.array(I.GROUNDED_CAVITY.box)
    assert xyz.shape == (20_000, 3) and q.sum() == 0
    assert np.all(xyz >= 0.05) and np.all(xyz <= L - 0.05)
    assert I.GROUNDED_CAVITY.R == np.sqrt(3.0) * 0.5 * np.linalg.norm(L)


def test_pm1_sizes_round_up_to_even_and_stay_neutral():
    for n in (1, 2, 3, 257, 1001):
        xyz, q = I.uniform_pm1(n, (1.0, 1.3, 0.8), seed_offset=9)
        assert len(q) == n + n % 2 and q.sum() == 0 and xyz.shape == (len(q), 3)
        assert np.all(xyz < np.array([1.0, 1.3, 0.8]))


def test_batch_and_serving_size_distributions():
    systems = I.batch_periodic()
    sizes = np.array([len(s[1]) for s in systems])
    assert len(systems) == 256 and np.all(sizes % 2 == 0)
    assert sizes.min() >= 500 and sizes.max() <= 50_000
    # log-uniform: the median of log N sits near the middle of [log 500, log 50000]
    assert abs(np.median(np.log(sizes)) - 0.5 * (np.log(500) + np.log(50_000))) < 0.4
    assert all(abs(s[1].sum()) == 0 for s in systems)
    t, n = I.poisson_trace(2000)
    assert t[0] == 0 and np.all(np.diff(t) >= 0)
    assert abs(len(t) / t[-1] - 2000.0) < 150.0  # arrival rate 2000/s
    assert n.min() >= 1000 and n.max() <= 200_000 and np.all(n % 2 == 0)


def test_lattices():
    xyz, q = I.nacl_lattice(4, 2.0)
    assert xyz.shape == (64, 3) and q.sum() == 0
    # nearest neighbours carry opposite charges
    d = np.linalg.norm(xyz[:, None] - xyz[None], axis=-1)
    nn = np.isclose(d, 0.5)
    assert np.all((q[:, None] * q[None])[nn] == -1)
    xyz, q = I.lattice_random_sign(5)
    assert xyz.shape == (125, 3) and q.sum() == 0 and np.count_nonzero(q == 0) == 1
    xyz, q = I.lattice_random_sign(6)
    assert q.sum() == 0 and np.count_nonzero(q == 0) == 0


def test_generators_are_deterministic_in_their_seed():
    a = I.uniform_gauss(500, (1.0, 1.0, 1.0), seed_offset=3)
    b = I.uniform_gauss(500, (1.0, 1.0, 1.0), seed_offset=3)
    c = I.uniform_gauss(500, (1.0, 1.0, 1.0), seed_offset=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    assert I.rng(0).integers(1 << 62) == np.random.default_rng(1806_04801).integers(1 << 62)
