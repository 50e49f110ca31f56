"""Pins of the overlap-signature basis order (oracle/reorder.py) and the
library's host implementation (kldi_order_shells) against it; no GPU."""
import numpy as np
import pytest

import synth
from oracle import reorder as orr


def test_merge_heights_equal_scipy_average_linkage():
    hier = pytest.importorskip("scipy.cluster.hierarchy")
    dist = pytest.importorskip("scipy.spatial.distance")
    rng = np.random.default_rng(4)
    X = rng.normal(size=(40, 5))
    d0 = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    h = []
    orr.cluster_order(d0, h)
    Z = hier.linkage(dist.squareform(d0, checks=False), method="average")
    assert np.allclose(np.sort(h), np.sort(Z[:, 2]), rtol=1e-12, atol=0)


def test_points_on_a_line_come_out_monotonic():
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 100, size=60)
    d0 = np.abs(x[:, None] - x[None, :])
    order = orr.cluster_order(d0)
    xs = x[order]
    assert np.all(np.diff(xs) > 0) or np.all(np.diff(xs) < 0)


def test_separate_molecules_form_contiguous_segments():
    s = synth.make_system(1)                         # two waters, 3 A apart
    far = s.xyz.copy()
    far[3:] += np.array([200.0, 0.0, 0.0])           # move the second water out of overlap range
    b = s.basis
    S = synth.overlap_matrix(far, b)
    perm = orr.order_shells(S, synth.shell_sizes(b))
    mol = (b.atom[perm] >= 3).astype(int)
    assert np.count_nonzero(np.diff(mol)) == 1
    assert sorted(perm.tolist()) == list(range(b.nshell))


@pytest.mark.parametrize("name", ["w1", "w4", "w33"])
def test_library_order_equals_oracle(name):
    from paper_2605_10363_gb300 import kldi
    s = synth.make_system(1) if name == "w1" else synth.make_system(2, nwaters=None if name == "w33" else 4)
    S = synth.overlap_matrix(s.xyz, s.basis)
    nfn = synth.shell_sizes(s.basis)
    assert np.array_equal(kldi.order_shells(S, nfn), orr.order_shells(S, nfn))


def test_library_order_rejects_bad_input():
    from paper_2605_10363_gb300 import kldi
    with pytest.raises(ValueError):
        kldi.order_shells(np.eye(3), np.array([1, 1]))
    with pytest.raises(kldi.KldiError) as e:
        kldi.order_shells(np.eye(3), np.array([1, 0, 2]))
    assert e.value.status == kldi.EINVAL
    with pytest.raises(kldi.KldiError):
        kldi.order_shells(np.zeros((2, 2)), np.array([1, 1]))   # zero signatures
