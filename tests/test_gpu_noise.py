"""The device's PILE_L noise (App. D: eta ~ N(0, 1) per mode, atom and step)
against the oracle: Philox-4x32-10 words bit for bit over a grid of (seed,
stream, step, mode, atom), and the FP64 Box-Muller deviates within 8 ulp of
the Box-Muller radius of the oracle's.  Both sides evaluate log, sqrt, sin and
cos in FP64 with different libraries; the oracle rounds the angle 2 pi u
before its cosine (an absolute error up to ~3.5 ulp of 1, times a radius of up
to ~6.7) where the device calls sincospi(2 u), so the deviates may differ by
about 5 ulp of the radius but no more."""
import numpy as np
import pytest

from tests._gpu import pimd  # noqa: F401
from tests._kat import published_vectors

pytestmark = pytest.mark.gpu

GRID = [(1, 0, 0), (1, 0, 99), (1, 1, 100), (1, 2, 0), (7, 0, 2**32 + 5), (0x0123456789ABCDEF, 3, 12345),
        (2**63 + 11, 1, 2**40 - 1)]


@pytest.mark.parametrize("seed,stream,step", GRID)
def test_noise_words_and_deviates(orc, pimd, seed, stream, step):
    n_atoms, n_modes = 37, 33   # ragged: neither a multiple of a warp
    words, eta = pimd.noise_sample(seed, stream, step, n_atoms, n_modes)
    for k in range(n_modes):
        for i in range(n_atoms):
            ctr = [i, (k & 0xFFFF) | (stream << 16), step & 0xFFFFFFFF, step >> 32]
            want = orc.philox4(32, 10, ctr, [seed & 0xFFFFFFFF, seed >> 32])
            assert list(map(int, words[k, i])) == list(map(int, want)), (k, i)
            c = orc.gauss3(seed, i, k, stream, step)
            # the radius sqrt(-2 ln u) sets the scale of each deviate's rounding
            u = (words[k, i].astype(np.float64) + 0.5) * 2.0**-32
            r = np.sqrt(-2.0 * np.log(u[[0, 0, 2]]))
            tol = 8 * np.spacing(np.maximum(r, 1.0))
            assert np.all(np.abs(eta[k, i] - c) <= tol), (k, i, eta[k, i], c)


def test_device_words_match_published_vector(pimd):
    """The published all-zero Philox-4x32-10 vector (counter 0, key 0) is the
    device's word for seed 0, atom 0, mode 0, stream 0, step 0."""
    ctr, key, out = published_vectors()[0]
    assert ctr == [0, 0, 0, 0] and key == [0, 0]
    words, _ = pimd.noise_sample(0, 0, 0, 1, 1)
    assert list(map(int, words[0, 0])) == out
