"""The seeded input generators (CPU): determinism, statistics, and the
counter-based generator's independence across arrays and seeds."""
import numpy as np

from paper_1201_5029_gb300 import inputs as I


def test_white_ics_are_seeded_and_shaped():
    w = I.workload("preheat32")
    a = I.initial_fields(w, n=8)
    b = I.initial_fields(w, n=8)
    assert a[0].shape == (2, 8, 8, 8) and np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert abs(np.mean(a[0][0]) - 1.0) < 1e-5 and abs(np.mean(a[1][0]) + 0.5) < 1e-5


def test_spectral_ics_rms_and_zero_mode():
    w = I.workload("preheat128")
    phi, pi = I.initial_fields(w, n=16)
    for f in range(2):
        d = phi[f] - w["background"][f]
        assert abs(np.sqrt(np.mean(d * d)) - w["noise"]) < 1e-12
        assert abs(np.mean(d)) < 1e-17


def test_philox_normals_statistics_and_independence():
    z = I.philox_normals(12345, 0, 200000)
    assert abs(np.mean(z)) < 0.01 and abs(np.var(z) - 1.0) < 0.01
    assert abs(np.mean(z ** 3)) < 0.03 and abs(np.mean(z ** 4) - 3.0) < 0.05
    z2 = I.philox_normals(12345, 1, 200000)
    z3 = I.philox_normals(12346, 0, 200000)
    assert abs(np.corrcoef(z, z2)[0, 1]) < 0.01 and abs(np.corrcoef(z, z3)[0, 1]) < 0.01
    assert np.array_equal(z[:1000], I.philox_normals(12345, 0, 1000))


def test_philox_round_function_is_a_bijection_on_a_sample():
    """Different counters give different outputs (no collisions on a sample)."""
    c = np.arange(100000, dtype=np.uint64)
    out = I.philox4x32_10(c, np.zeros_like(c), np.zeros_like(c), np.zeros_like(c), 7, 9)
    packed = (out[0] << np.uint64(32)) | out[1]
    assert len(np.unique(packed)) == len(c)
