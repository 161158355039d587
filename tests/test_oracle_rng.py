"""Pins of the oracle's Philox generator (Salmon et al., SC'11) and of the
Box-Muller Gaussian noise used by the PILE_L O step (App. D)."""
import math

import numpy as np
import pytest
from scipy import stats

from tests._kat import published_vectors


def test_philox4x32_10_published_vectors(orc):
    """The oracle's Philox-4x32-10 reproduces the generator's published
    known-answer vectors (no library or interpreter involved)."""
    rows = published_vectors()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert list(map(int, orc.philox4(32, 10, ctr, key))) == out, (ctr, key)


def test_philox_4x64_matches_numpy(orc):
    """numpy's Philox bit generator is Philox-4x64-10 and emits block i from
    counter i+1.  The oracle's generic Philox (same code path as the 4x32
    variant used by the method) must reproduce it word for word."""
    for key in (0, 1, 0x0123456789ABCDEF):
        bg = np.random.Philox(key=key, counter=0)
        raw = bg.random_raw(4 * 5)
        for blk in range(5):
            out = orc.philox4(64, 10, [blk + 1, 0, 0, 0], [key & (2**64 - 1), 0])
            assert list(map(int, out)) == list(map(int, raw[4 * blk:4 * blk + 4]))


def test_philox_weyl_constants_from_definition(orc):
    """The key schedule adds floor(2^w (phi - 1)) and floor(2^w (sqrt 3 - 1)).
    With a zero counter and zero multiplier input the round function reduces to
    XORs of the key, so two rounds expose the bumped key."""
    for w in (32, 64):
        one = 1 << w
        phi_frac = (math.isqrt(5 * one * one) - one) // 2      # floor(2^w (sqrt5 - 1)/2)
        s3 = math.isqrt(3 * one * one) - one                     # floor(2^w (sqrt3 - 1))
        # first Philox round with ctr = 0: hi/lo of products are 0 -> c = (k0, 0, k1, 0)
        # second Philox round (key bumped): checked through the one-round identity instead
        out1 = orc.philox4(w, 1, [0, 0, 0, 0], [0, 0])
        assert list(map(int, out1)) == [0, 0, 0, 0]
        # with ctr zero and key K, one round gives (k0, 0, k1, 0)
        out1 = orc.philox4(w, 1, [0, 0, 0, 0], [5, 7])
        assert list(map(int, out1)) == [5, 0, 7, 0]
        # two rounds from ctr zero, key zero: second round sees c = (0,0,0,0) and
        # the bumped key (W0, W1), so it returns (W0, 0, W1, 0)
        out2 = orc.philox4(w, 2, [0, 0, 0, 0], [0, 0])
        assert int(out2[0]) == phi_frac and int(out2[2]) == s3
        assert int(out2[1]) == 0 and int(out2[3]) == 0


def _eta(orc, n_atoms, modes, steps, seed=7, stream=0):
    out = []
    for s in steps:
        for k in modes:
            for i in range(n_atoms):
                out.append(orc.gauss3(seed, i, k, stream, s))
    return np.array(out)


def test_gauss_distribution(orc):
    eta = _eta(orc, 200, range(8), range(40))      # 64000 x 3 draws
    flat = eta.ravel()
    n = flat.size
    assert abs(flat.mean()) < 5 / math.sqrt(n)
    assert abs(flat.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(stats.skew(flat)) < 5 * math.sqrt(6.0 / n)
    assert abs(stats.kurtosis(flat)) < 5 * math.sqrt(24.0 / n)
    for a in range(3):
        assert stats.kstest(eta[:, a], "norm").pvalue > 1e-4


def test_gauss_independence(orc):
    """No correlation between components, adjacent atoms, modes, steps, seeds
    or streams."""
    n = 4000
    base = np.array([orc.gauss3(3, i, 1, 0, 10) for i in range(n)])
    nxt_atom = np.array([orc.gauss3(3, i + 1, 1, 0, 10) for i in range(n)])
    nxt_mode = np.array([orc.gauss3(3, i, 2, 0, 10) for i in range(n)])
    nxt_step = np.array([orc.gauss3(3, i, 1, 0, 11) for i in range(n)])
    nxt_seed = np.array([orc.gauss3(4, i, 1, 0, 10) for i in range(n)])
    nxt_strm = np.array([orc.gauss3(3, i, 1, 1, 10) for i in range(n)])
    bound = 5.0 / math.sqrt(n)
    for other in (nxt_atom, nxt_mode, nxt_step, nxt_seed, nxt_strm):
        for a in range(3):
            assert abs(np.corrcoef(base[:, a], other[:, a])[0, 1]) < bound
    c = np.corrcoef(base.T)
    assert np.abs(c - np.eye(3)).max() < bound


def test_gauss_large_step_counter(orc):
    """The step counter spans 64 bits: steps 2^32 apart differ."""
    a = orc.gauss3(1, 0, 0, 0, 5)
    b = orc.gauss3(1, 0, 0, 0, 5 + (1 << 32))
    assert not np.allclose(a, b)
