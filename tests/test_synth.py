"""The seeded generator: reproducible, slice-consistent, thread-count independent, in range."""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reproducible_and_slice_consistent():
    w = synth.workload("voigt_1e7").scaled(n_trans=50_000)
    a = w.transitions()
    b = w.transitions(20_000, 10_000)
    for x, y in zip(a, b):
        assert np.array_equal(x[20_000:30_000], y)
    assert all(np.array_equal(x, y) for x, y in zip(a, w.transitions()))


def test_ids_and_ranges():
    for name in ("doppler_1e5", "voigt_1e7", "voigt_1e9"):
        w = synth.workload(name).scaled(n_trans=20_000, n_states=min(synth.workload(name).n_states, 2_000_000))
        up, lo, A = w.transitions()
        ns = w.n_states
        assert up.min() >= 0 and up.max() < ns and lo.min() >= 0 and lo.max() < ns
        assert A.min() >= 10 ** w.logA[0] * 0.999 and A.max() <= 10 ** w.logA[1] * 1.001
        gr, ne = w.broadening()
        assert gr.min() >= 0.03 and gr.max() <= 0.1 and ne.min() >= 0.4 and ne.max() <= 0.8


def test_level_schemes():
    w = synth.workload("doppler_1e5")
    E, g, Ev = w.states()
    assert E.size == 5000 and E[0] == 0.0 and g[0] == 3 and g[1] == 9
    J = 70
    assert abs(E[J] - (10 * J * (J + 1) - 1e-3 * (J * (J + 1)) ** 2)) < 1e-9
    assert np.all(np.diff(E[:1000]) > 0)       # clamped law keeps increasing
    El, _, _ = w.states(literal=True)
    assert El[999] < -1e8                        # the literal quartic turns negative
    p = synth.workload("voigt_1e9").scaled(n_states=20_000)
    E, g, Ev = p.states()
    assert np.all(g >= 1) and np.all(g % 2 == 1) and np.all(Ev >= 0) and np.all(E >= Ev - 1e-9)


def test_thread_count_independent():
    code = ("import sys; sys.path.insert(0, %r); import synth, hashlib; w = synth.workload('voigt_1e9')"
            ".scaled(n_trans=200000, n_states=1000000); u, l, A = w.transitions();"
            "print(hashlib.sha256(u.tobytes() + l.tobytes() + A.tobytes()).hexdigest())" % ROOT)
    outs = []
    for t in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=t)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                                   check=True).stdout.strip())
    assert outs[0] == outs[1]


def test_vibronic_densities_are_per_manifold_normalised_and_seeded():
    w = synth.workload("nlte_1e7")
    d = w.vib_densities()
    assert d.shape == (w.n_states,) and d.dtype == np.float64
    per_v = d.reshape(w.nv, w.nJ)
    assert np.all(per_v == per_v[:, :1])                     # one weight per vibrational manifold
    assert per_v[:, 0].sum() == pytest.approx(1.0, rel=1e-14)
    assert np.all(per_v[:, 0] > 0) and np.array_equal(d, w.vib_densities())
    with pytest.raises(ValueError):
        synth.workload("voigt_1e9").vib_densities()
