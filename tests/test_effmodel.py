"""Host logic of the effective-model class tables (Eq. 2; the 16-coupling
model and the range scans of "Results"), checked against the oracle's
features on CPU."""
import numpy as np

from oracle import oracle as O
from paper_1612_03804_gb300 import effmodel as E
from paper_1612_03804_gb300.inputs import uniform_field


def test_paper_model_has_sixteen_couplings_within_the_library_limits():
    cls = E.paper_classes()
    assert len(cls) == 16 and len(E.class_names()) == 16
    assert E.n_offsets(cls) <= 64 and len(cls) <= 32
    kinds = [(sum(o[2] == 0 for o in c) == len(c), all(o[:2] == (0, 0) for o in c)) for c in cls]
    assert sum(1 for sp, tm in kinds if sp) == 2          # equal-slice classes
    assert sum(1 for sp, tm in kinds if tm) == 10         # same-site classes
    assert sum(1 for sp, tm in kinds if not sp and not tm) == 4


def test_each_unordered_pair_appears_once():
    for c in E.paper_classes(n_shell=5, n_time=10, st_shells=2, st_times=3):
        offs = set(c)
        for o in c:
            assert tuple(-x for x in o) not in offs or o == (0, 0, 0)
        assert len(offs) == len(c)


def test_shell_distances_grow():
    d = [min(dx * dx + dy * dy for dx, dy in sh) for sh in E.SHELLS]
    assert d == sorted(d) and len(set(d)) == len(d)
    for sh in E.SHELLS:
        assert len({dx * dx + dy * dy for dx, dy in sh}) == 1


def test_feature_counts_on_the_ordered_field():
    """All +1: f_c = number of (site, offset) pairs = V * |c| (no self-pairs at L=8, M=20)."""
    m = O.Model(8, 8, beta=1.0, dtau=0.05)
    s = np.ones((m.M, m.N), dtype=np.int8)
    cls = E.paper_classes()
    f = O.features(m, s, cls)
    np.testing.assert_array_equal(f, [m.M * m.N * len(c) for c in cls])


def test_temporal_features_are_lag_sums():
    """f for the temporal class k is the lag-k autocorrelation sum of the field."""
    m = O.Model(4, 3, beta=1.0, dtau=0.1)
    s = uniform_field(5, m.M, m.N)
    for k in (1, 3, 5):
        f = O.features(m, s, [E.temporal_class(k)])[0]
        assert f == int(np.sum(s.astype(np.int64) * np.roll(s, -k, axis=0)))


def test_range_scans():
    t = E.temporal_range_scan(10)
    assert [k for k, _ in t] == list(range(1, 11)) and len(t[-1][1]) == 11
    sp = E.spatial_range_scan(5)
    assert [s for s, _ in sp] == [1, 2, 3, 4, 5] and len(sp[-1][1]) == 15
