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


def _cells(d, p, keep):
    """Box indices (x fastest) of the cells c of a (p+2)^d box with keep(c)."""
    ne = p + 2
    return [sum(c[m] * ne ** m for m in range(d))
            for c in itertools.product(range(ne), repeat=d) if keep(c)]


def _span(idx):
    return max(idx) - min(idx) + 1


def _interior(p):
    return lambda c: all(1 <= x <= p for x in c)


def _read(p):  # interior and face-halo cells: at most one coordinate on the halo
    return lambda c: sum(1 for x in c if x in (0, p + 1)) <= 1


@pytest.mark.parametrize("d,p", [(1, 4), (2, 5), (2, 17), (3, 3), (3, 5), (3, 7)])
def test_copied_back_covers_the_interior(bench, d, p):
    """1D/2D: one span from the first to the last interior cell; 3D: one span
    per interior z-plane (x fastest, z the slowest coordinate)."""
    s = d + 2
    if d < 3:
        want = _span(_cells(d, p, _interior(p)))
    else:
        want = sum(_span(_cells(d, p, lambda c, z=z: _interior(p)(c) and c[2] == z))
                   for z in range(1, p + 1))
    assert bench._copied_back(d, p, s) == want * s


@pytest.mark.parametrize("d,p", [(1, 4), (2, 5), (2, 17), (3, 3), (3, 5), (3, 7)])
def test_copied_in_covers_what_the_update_reads(bench, d, p):
    """One span from the first to the last face-halo cell."""
    s = d + 2
    assert bench._copied_in(d, p, s) == _span(_cells(d, p, _read(p))) * s


def test_copied_5cubed_counts(bench):
    """5^3 boxes (343 cells): 327 cells in, 165 back (one span back would
    take 229)."""
    assert bench._copied_in(3, 5, 1) == 327
    assert bench._copied_back(3, 5, 1) == 165


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


def test_issue_roofline_uses_the_committed_count_only_for_its_kernel(bench, monkeypatch):
    """The correction kernel's issue roofline: warp instructions per launch over
    one warp instruction per scheduler per clock (4 x 152 SMs x 2.07 GHz); no
    figure on another mesh, or once the kernel's sources differ from those the
    count was taken on."""
    monkeypatch.setattr(bench, "_warp_instructions", lambda key: 1.25856e9)
    r = bench._issue_roofline(1.0, 1024)  # 1.25856e9 instructions in 1 ms: the peak rate
    assert r["bound"] == "issue"
    assert r["peak"] == pytest.approx(4 * 152 * 2.07e9 / 1e12)
    assert r["frac"] == pytest.approx(1.0)
    assert bench._issue_roofline(1.0, 512) is None
    monkeypatch.setattr(bench, "_warp_instructions", lambda key: None)
    assert bench._issue_roofline(1.0, 1024) is None


def test_committed_counts_are_keyed_by_kernel_hash(bench, monkeypatch):
    """A count taken on other sources is not used."""
    from paper_2302_09005_gb300 import _build
    assert bench._warp_instructions("corr_shear_1024") == 92208896
    monkeypatch.setattr(_build, "kernel_hash", lambda kind="step": "0" * 16)
    assert bench._warp_instructions("corr_shear_1024") is None
    assert bench._traffic("euler3d_fp32_262144x5") is None
