"""Mixed batch in the oracle: the per-event row rule and the identity of every
event with the one-process run of its row."""
import numpy as np
import pytest

from oracle import oracle as O

FRACTIONS = [0.5, 0.25, 0.25]


def _rows():
    return [O.Settings(process=2, sqrt_s=13600.0, t_cut=1.0, nmax=128, seed=1),
            O.Settings(process=0, sqrt_s=91.2, t_cut=0.5, nmax=128, seed=1),
            O.Settings(process=0, sqrt_s=500.0, t_cut=4.0, nmax=128, seed=1)]


def test_row_rule_restated_from_philox():
    """Row = first cumulative share above the uniform of block (seed, id, 2^62),
    computed here from the Philox and uniform primitives."""
    seed, first = 7, (1 << 33) + 5
    rows = O.mix_rows(seed, FRACTIONS, first, 400)
    cum = np.cumsum(FRACTIONS)
    for i in range(400):
        e = first + i
        w = O.philox([e & 0xFFFFFFFF, e >> 32, 0, 1 << 30], [seed & 0xFFFFFFFF, seed >> 32])
        u = O.uniform(w[0], w[1])
        expect = next((k for k in range(len(cum) - 1) if u < cum[k]), len(cum) - 1)
        assert rows[i] == expect


def test_row_shares_are_binomial():
    n = 200_000
    rows = O.mix_rows(1, FRACTIONS, 0, n)
    for k, f in enumerate(FRACTIONS):
        c = int((rows == k).sum())
        assert abs(c - n * f) < 5 * np.sqrt(n * f * (1 - f))


def test_single_row_is_the_plain_run(pdf):
    st = O.Settings(process=0, sqrt_s=91.2, nmax=128, seed=1)
    a = O.run_mix([st], [1.0], 100, 200)
    b = O.run(st, 100, 200)
    assert np.all(a["row"] == 0)
    for k in ("p", "flav", "weight", "obs", "npart"):
        assert np.array_equal(a[k], b[k])


def test_mixed_events_equal_their_row_runs(pdf):
    rows = _rows()
    first, n = 1000, 300
    mix = O.run_mix(rows, FRACTIONS, first, n, pdf, threads=4)
    assert set(np.unique(mix["row"])) == {0, 1, 2}
    for r, st in enumerate(rows):
        ref = O.run(st, first, n, pdf if st.process else None, threads=4)
        sel = mix["row"] == r
        for k in ("p", "flav", "col", "acol", "npart", "status", "weight", "obs", "counters"):
            assert np.array_equal(mix[k][sel], ref[k][sel]), (r, k)


def test_bad_tables_are_rejected(pdf):
    with pytest.raises(RuntimeError):
        O.run_mix([O.Settings(seed=1), O.Settings(seed=2)], [0.5, 0.5], 0, 10)
