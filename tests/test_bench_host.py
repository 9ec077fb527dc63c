"""Host-side accounting of bench.py (no GPU): the spans the in-place host
pipeline copies in and back, against the cells of a patch box counted one by
one, and the algorithmic bytes per patch of the roofline."""
import importlib.util
import itertools
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("d,p", [(1, 4), (2, 5), (2, 17), (3, 3), (3, 5), (3, 7)])
def test_interior_span_is_first_to_last_interior_cell(bench, d, p):
    s = d + 2
    ne = p + 2
    idx = [sum(c[m] * ne ** m for m in range(d))
           for c in itertools.product(range(ne), repeat=d) if all(1 <= x <= p for x in c)]
    assert bench._interior_span(d, p, s) == (max(idx) - min(idx) + 1) * s


@pytest.mark.parametrize("d,p", [(1, 4), (2, 5), (2, 17), (3, 3), (3, 5), (3, 7)])
def test_face_halo_span_covers_what_the_update_reads(bench, d, p):
    s = d + 2
    ne = p + 2
    idx = [sum(c[m] * ne ** m for m in range(d))
           for c in itertools.product(range(ne), repeat=d)
           if sum(1 for x in c if x in (0, p + 1)) <= 1]  # interior and face-halo cells
    assert bench._face_halo_span(d, p, s) == (max(idx) - min(idx) + 1) * s


@pytest.mark.parametrize("d,p", [(2, 5), (3, 5), (3, 7)])
def test_algorithmic_bytes_count_interior_and_face_halo(bench, d, p):
    s, item = d + 2, 4
    interior = p ** d
    face_halo = 2 * d * p ** (d - 1)
    assert bench.alg_bytes_per_patch(d, p, item) == ((interior + face_halo) * s + interior * s) * item


def test_equal_cost_interpolation(bench):
    """Plain cost growing as N^3 and error as N^-1.5: the resolution whose cost
    is twice the N = 1000 cost is 1000 * 2^(1/3), and the error there follows
    the same power law (both exact in log-log)."""
    cost = {n: 0.5 * (n / 1000.0) ** 3 for n in (1000, 1400, 2000)}
    err = {n: 3e-3 * (n / 1000.0) ** -1.5 for n in (1000, 2000)}
    r = bench._equal_cost(cost, err, 1.0)
    assert r["N_at_learned_cost"] == pytest.approx(1000 * 2 ** (1 / 3), rel=1e-12)
    assert r["plain_mean_rel_l1"] == pytest.approx(3e-3 * 2 ** -0.5, rel=1e-12)
    assert r["interpolated"]
    # outside the timed range: extrapolated from the end segment, and said so
    r = bench._equal_cost(cost, err, 0.25)
    assert r["N_at_learned_cost"] == pytest.approx(1000 * 0.5 ** (1 / 3), rel=1e-12)
    assert not r["interpolated"]
