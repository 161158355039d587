"""Known-answer pin of the oracle's Philox-4x32-10 (Salmon, Moraes, Dror and
Shaw, SC'11) and of the noise keying the PILE_L O step draws from (App. D's
eta ~ N(0, 1), independent per mode, atom and step).

The answers come from an implementation the oracle shares nothing with:
Triton's ``tl.random.philox`` library routine (round multipliers 0xD2511F53 and
0xCD9E8D57, Weyl key increments, ten rounds; a 64-bit seed becomes the key
(seed low 32 bits, seed high 32 bits)), executed on the CPU by Triton's
interpreter in a child process, so no GPU and no compiled Triton kernel is
involved.  A wrong round multiplier, a swapped output word, a missing key bump
or a different key split in ``oracle/pimd_oracle.c`` changes every word and
fails here; the statistical tests in test_oracle_rng.py cannot see a wrong
constant that still mixes well.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytest.importorskip("triton")

_CHILD = r"""
import json, sys
import numpy as np
import torch
import triton
import triton.language as tl

@triton.jit
def _words(seed_ptr, ctr_ptr, out_ptr, n, BLOCK: tl.constexpr):
    i = tl.arange(0, BLOCK)
    m = i < n
    seed = tl.load(seed_ptr + i, mask=m)
    c0 = tl.load(ctr_ptr + 4 * i + 0, mask=m)
    c1 = tl.load(ctr_ptr + 4 * i + 1, mask=m)
    c2 = tl.load(ctr_ptr + 4 * i + 2, mask=m)
    c3 = tl.load(ctr_ptr + 4 * i + 3, mask=m)
    o0, o1, o2, o3 = tl.random.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + 4 * i + 0, o0.to(tl.int32, bitcast=True), mask=m)
    tl.store(out_ptr + 4 * i + 1, o1.to(tl.int32, bitcast=True), mask=m)
    tl.store(out_ptr + 4 * i + 2, o2.to(tl.int32, bitcast=True), mask=m)
    tl.store(out_ptr + 4 * i + 3, o3.to(tl.int32, bitcast=True), mask=m)

cases = json.load(sys.stdin)
n = len(cases)
block = 1
while block < n:
    block *= 2
seeds = torch.tensor(np.array([c[0] for c in cases], dtype=np.uint64).view(np.int64))
ctr = torch.tensor(np.array([c[1] for c in cases], dtype=np.uint32).view(np.int32))
out = torch.zeros((n, 4), dtype=torch.int32)
_words[(1,)](seeds, ctr, out, n, BLOCK=block)
json.dump(out.numpy().view(np.uint32).tolist(), sys.stdout)
"""


def _library_words(cases):
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _CHILD], input=json.dumps(cases), env=env,
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("Triton interpreter unavailable: " + r.stderr.strip().splitlines()[-1])
    return json.loads(r.stdout)


def _cases():
    rng = np.random.default_rng(20260213)
    m32 = 0xFFFFFFFF
    cases = [
        (0, [0, 0, 0, 0]),
        (2**64 - 1, [m32, m32, m32, m32]),
        (1, [0, 0, 0, 0]),
        (1, [191, 31, 9999, 0]),
        (0x0123456789ABCDEF, [5, (7 & 0xFFFF) | (1 << 16), 123456, 1]),
        (2**32, [0, 0, 0, 0]),           # key (0, 1): the high seed word alone
        (7, [0xFFFFFFFF, (3 << 16) | 0xFFFF, m32, m32]),   # the barostat's atom word
    ]
    for _ in range(57):
        seed = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        ctr = [int(v) for v in rng.integers(0, 2**32, size=4, dtype=np.uint64)]
        cases.append((seed, ctr))
    return cases


def test_philox4x32_10_known_answers(orc):
    """The oracle's generic Philox at w = 32, ten rounds, word for word."""
    cases = _cases()
    want = _library_words(cases)
    for (seed, ctr), w in zip(cases, want):
        got = orc.philox4(32, 10, ctr, [seed & 0xFFFFFFFF, seed >> 32])
        assert list(map(int, got)) == w, (seed, ctr)


def test_noise_keying_known_answers(orc):
    """The method's keying -- key (seed lo, seed hi), counter (atom, mode |
    stream << 16, step lo, step hi) -- and the Box-Muller map u = (w + 1/2)
    2^-32, (eta_x, eta_y) = sqrt(-2 ln u0) (cos, sin)(2 pi u1), eta_z =
    sqrt(-2 ln u2) cos(2 pi u3), evaluated on the library's words, against
    the oracle's deviates (the same double-precision functions on both sides:
    equal to the last few ulp)."""
    rng = np.random.default_rng(7)
    keys = [(1, 0, 0, 0, 0), (1, 191, 31, 0, 9999), (3, 5, 63, 1, 2**32 + 17),
            (2**40 + 3, 0xFFFFFFFF, 0, 3, 12), (9, 1, 127, 2, 0)]
    for _ in range(40):
        keys.append((int(rng.integers(1, 2**62)), int(rng.integers(0, 12288)),
                     int(rng.integers(0, 128)), int(rng.integers(0, 3)), int(rng.integers(0, 2**40))))
    cases = [(s, [a, (k & 0xFFFF) | (st << 16), n & 0xFFFFFFFF, n >> 32]) for s, a, k, st, n in keys]
    words = _library_words(cases)
    for (s, a, k, st, n), w in zip(keys, words):
        u = (np.array(w, dtype=np.float64) + 0.5) * 2.0**-32
        r0, r1 = np.sqrt(-2.0 * np.log(u[0])), np.sqrt(-2.0 * np.log(u[2]))
        want = np.array([r0 * np.cos(2 * np.pi * u[1]), r0 * np.sin(2 * np.pi * u[1]),
                         r1 * np.cos(2 * np.pi * u[3])])
        got = orc.gauss3(s, a, k, st, n)
        assert np.all(np.abs(got - want) <= 8 * np.spacing(np.maximum(np.abs(want), 1.0))), (s, a, k, st, n)
