"""Pins of the counter-based generator that the CUDA library uses to draw the setup's random
test vectors (the seeded inputs of Alg. 3); synth implements the same steps so that the
oracle can be fed the identical fields.

* Philox4x32-10 against its published known-answer values (tests/golden);
* the series logarithm, sine and cosine against numpy's library routines (a wrong
  coefficient, term count or quadrant would show far above 1e-15);
* the Box-Muller output against the N(0, 1) moments;
* the counter layout: fields, levels and seeds give different streams, and a field's
  entries do not depend on how many fields are drawn with it.
"""
import os

import numpy as np

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            w = [int(t, 16) for t in ln.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        got = synth.philox4x32_10(*ctr, *key)
        assert [int(g) for g in got] == out


def test_philox_vectorised_equals_scalar():
    c = np.arange(5, dtype=np.uint64)
    vec = synth.philox4x32_10(c, 7, 11, 13, 0x1234, 0x5678)
    for i in range(5):
        one = synth.philox4x32_10(i, 7, 11, 13, 0x1234, 0x5678)
        assert all(int(v[i]) == int(o) for v, o in zip(vec, one))


def test_series_log_and_trig_match_library_routines():
    rng = np.random.default_rng(3)
    u = np.concatenate([rng.random(200000), [2.0 ** -53, 0.5, 0.7071067811865476, 1.0 - 2.0 ** -53, 1.0]])
    u = u[u > 0]
    ref = np.log(u)
    got = synth._ln(u)
    assert np.all(np.abs(got - ref) <= 2e-15 * np.maximum(1.0, np.abs(ref)))
    assert synth._ln(np.array([1.0]))[0] == 0.0
    v = np.concatenate([rng.random(200000), [0.0, 0.25, 0.5, 0.75, 0.125, 0.999999]])
    s, c = synth._sincos_2pi(v)
    assert np.max(np.abs(s - np.sin(2 * np.pi * v))) <= 2e-15
    assert np.max(np.abs(c - np.cos(2 * np.pi * v))) <= 2e-15
    assert np.max(np.abs(s * s + c * c - 1.0)) <= 4e-16 * 8


def test_normal_moments():
    f = synth.philox_fields(8, (8, 8, 8, 8), 12, 20240)
    x = np.concatenate([f.real.ravel(), f.imag.ravel()])
    n = x.size                                   # 786432 samples
    assert abs(x.mean()) < 5 / np.sqrt(n)
    assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(np.mean(x ** 4) - 3.0) < 5 * np.sqrt(96.0 / n)
    assert abs(np.mean(f.real * f.imag)) < 5 / np.sqrt(n / 2)   # real and imaginary parts independent


def test_counter_layout():
    a = synth.philox_fields(3, (2, 2, 2, 4), 12, 99)
    b = synth.philox_fields(1, (2, 2, 2, 4), 12, 99, j0=2)
    assert np.array_equal(a[2], b[0])                          # field j is the same drawn alone
    c = synth.philox_fields(1, (2, 2, 2, 4), 12, 99, level=1, j0=2)
    d = synth.philox_fields(1, (2, 2, 2, 4), 12, 100, j0=2)
    e = synth.philox_fields(1, (2, 2, 2, 4), 12, 99 + (1 << 32), j0=2)   # the seed's high word counts
    for other in (c, d, e):
        assert not np.any(other[0] == b[0])
    tv = synth.philox_test_vectors([(4, 4, 4, 4), (2, 2, 2, 2)], (3, 5), 7)
    assert tv[0].shape == (3, 4, 4, 4, 4, 12) and tv[1].shape == (2, 2, 2, 2, 2, 6)
    assert np.array_equal(tv[1], synth.philox_fields(2, (2, 2, 2, 2), 6, 7, level=1))
