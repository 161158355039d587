"""The multi-replica batch engine (split precision): agreement with the FP64
oracle, bitwise independence of a replica from the rest of the batch,
per-replica step budgets, membership changes between runs, autotuning."""
import numpy as np
import pytest

from paper_2602_13553_gb300 import inputs
from tests._gpu import assert_split_close, pimd  # noqa: F401

pytestmark = pytest.mark.gpu


def rep(nmol, P, seed, T=300.0, deut=False):
    L = inputs.box_length(nmol)
    x0, mass = inputs.water_box(nmol, L, P, seed, jitter=0.02, deuterium=deut)
    return dict(x0=x0, mass=mass, T=T, dt=5e-4, ff=inputs.water_ff_for_box(L), box=(L, L, L), seed=seed)


def add(b, r, nsteps, **kw):
    return b.add(r["x0"], r["mass"], T=r["T"], dt=r["dt"], nsteps=nsteps, ff=r["ff"], box=r["box"],
                 seed=r["seed"], **kw)


MIX = [rep(40, 8, 11, 200.0), rep(70, 16, 12, 350.0, True), rep(100, 32, 13), rep(32, 64, 14, 120.0, True),
       rep(150, 8, 15, 390.0), rep(64, 32, 16)]


def test_batch_agrees_with_oracle(orc, pimd):
    b = pimd.Batch(8)
    slots = [add(b, r, 40) for r in MIX[:3]]
    b.run(40)
    for s, r in zip(slots, MIX[:3]):
        c = orc.Sim(r["x0"], r["mass"], T=r["T"], dt=r["dt"], potential=1, ff=r["ff"], box=r["box"],
                    seed=r["seed"])
        c.run(40)
        x, v, st = b.get_state(s)
        assert st == 40
        assert_split_close(x, v, b.estimators()[s], c, c.estimators(), "slot %d" % s)
    b.close()


def test_replica_alone_and_in_mix_are_bitwise_equal(pimd):
    alone = pimd.Batch(2)
    s0 = add(alone, MIX[2], 60)
    alone.run(60)
    xa, va, _ = alone.get_state(s0)
    ea = alone.estimators()[s0]
    mixed = pimd.Batch(8)
    slots = [add(mixed, r, 60) for r in MIX]
    mixed.run(60)
    xm, vm, _ = mixed.get_state(slots[2])
    em = mixed.estimators()[slots[2]]
    assert np.array_equal(xa, xm) and np.array_equal(va, vm)
    for k in ("H", "K_CV", "P_CV", "K_PR"):
        assert abs(ea[k] - em[k]) <= 1e-12 * abs(ea[k]), k


def test_step_budgets_per_replica(pimd):
    budgets = [13, 40, 77]
    b = pimd.Batch(4)
    slots = [add(b, r, n) for r, n in zip(MIX[:3], budgets)]
    b.run(50)
    b.run(50)
    st, left = b.status()
    for s, n in zip(slots, budgets):
        assert st[s] == n and left[s] == 0
    for s, r, n in zip(slots, MIX[:3], budgets):
        # same call boundaries: every run() ends with a closing half-kick
        solo = pimd.Batch(1)
        t = add(solo, r, n)
        solo.run(50)
        solo.run(50)
        xs, vs, _ = solo.get_state(t)
        xb, vb, _ = b.get_state(s)
        assert np.array_equal(xs, xb) and np.array_equal(vs, vb)


def test_membership_changes_between_runs(pimd):
    b = pimd.Batch(4)
    a = add(b, MIX[0], 1000)
    b.run(20)
    c = add(b, MIX[1], 40)
    b.run(20)
    b.remove(a)
    b.run(20)
    x, v, st = b.get_state(c)
    assert st == 40
    solo = pimd.Batch(1)
    t = add(solo, MIX[1], 40)
    solo.run(20)
    solo.run(20)
    xs, vs, _ = solo.get_state(t)
    assert np.array_equal(xs, x) and np.array_equal(vs, v)


def test_autotune_changes_no_trajectory(pimd):
    reps = MIX[:3]
    tuned = pimd.Batch(4)
    slots = [add(tuned, r, 200) for r in reps]
    tiles = tuned.autotune(1)
    st, _ = tuned.status()
    used = int(st[slots[0]])
    assert tiles.pop("warp_blocks_per_sm") >= 1
    assert set(tiles) == {8, 16, 32} and all(t >= 1 for t in tiles.values())
    tuned.run(30)
    plain = pimd.Batch(4)
    pslots = [add(plain, r, 200) for r in reps]
    plain.run(used)
    plain.run(30)
    for s, p in zip(slots, pslots):
        x1, v1, s1 = tuned.get_state(s)
        x2, v2, s2 = plain.get_state(p)
        assert s1 == s2 == used + 30
        assert np.array_equal(x1, x2) and np.array_equal(v1, v2)


def test_full_replica_mix_sampled_against_oracle(orc, pimd):
    """The 256-replica mix of the benchmark (32-512 molecules, P in {8, 16, 32,
    64}, T 100-400 K, H or D), autotuned launch shape as in bench.py, 20 steps;
    four replicas sampled across the mix (the largest, a P = 64, a P = 8 and a
    deuterated one) are compared with the oracle one by one."""
    reps = inputs.replica_mix(256, seed=1)
    b = pimd.Batch(256)
    systems = []
    for r in reps:
        x0, mass = inputs.water_box(r.nmol, r.L, r.P, r.seed, jitter=0.02, deuterium=r.deuterium)
        kw = dict(T=r.T, dt=5e-4, ff=inputs.water_ff_for_box(r.L), box=(r.L,) * 3, seed=r.seed)
        systems.append((x0, mass, kw))
        b.add(x0, mass, nsteps=10 ** 9, **kw)
    b.autotune(1)
    st0, _ = b.status()
    used = int(st0[0])
    b.run(20)
    picks = {max(range(256), key=lambda i: reps[i].nmol),
             next(i for i in range(256) if reps[i].P == 64),
             next(i for i in range(256) if reps[i].P == 8),
             next(i for i in range(256) if reps[i].deuterium and reps[i].P == 16)}
    est = b.estimators()
    for s in sorted(picks):
        x0, mass, kw = systems[s]
        c = orc.Sim(x0, mass, potential=1, **kw)
        c.run(used + 20)
        x, v, st = b.get_state(s)
        assert st == used + 20
        assert_split_close(x, v, est[s], c, c.estimators(), "replica %d" % s)
    b.close()


def test_batch_obabo_agrees_with_oracle(orc, pimd):
    """OBABO replicas (the merged closing B O / opening O B of the warp-item
    and block-item kernels, bead counts 8, 32 and 100) against the oracle."""
    b = pimd.Batch(4)
    reps = [MIX[0], MIX[2], rep(24, 100, 17, 250.0)]
    slots = [add(b, r, 40, integrator=1) for r in reps]
    b.run(25)
    b.run(15)
    for s, r in zip(slots, reps):
        c = orc.Sim(r["x0"], r["mass"], T=r["T"], dt=r["dt"], potential=1, ff=r["ff"], box=r["box"],
                    seed=r["seed"], integrator=1)
        c.run(40)
        x, v, st = b.get_state(s)
        assert st == 40
        assert_split_close(x, v, b.estimators()[s], c, c.estimators(), "OBABO P = %d" % r["x0"].shape[0])
    b.close()


@pytest.mark.parametrize("kw", [dict(sp=0.5), dict(thermostat=0), dict(tau=0.2, scale=0.5)])
def test_batch_keywords_agree_with_oracle(orc, pimd, kw):
    """Keywords that change only the mode tables or switch the thermostat
    (sp, NVE, tau and scale) in the batch engine, against the oracle."""
    b = pimd.Batch(2)
    r = MIX[1]
    s = add(b, r, 30, **kw)
    b.run(30)
    c = orc.Sim(r["x0"], r["mass"], T=r["T"], dt=r["dt"], potential=1, ff=r["ff"], box=r["box"],
                seed=r["seed"], **kw)
    c.run(30)
    x, v, st = b.get_state(s)
    assert st == 30
    assert_split_close(x, v, b.estimators()[s], c, c.estimators(), str(kw))
    b.close()


@pytest.mark.parametrize("integ", [0, 1])
def test_batch_128_beads_agree_with_oracle(orc, pimd, integ):
    """128-bead replicas (their own warp-item kernel, eight mode tiles) beside
    a 32-bead one and a 100-bead block-item one, BAOAB and OBABO, against the
    oracle; the 128-bead replica is bitwise the same alone."""
    b = pimd.Batch(4)
    reps = [rep(24, 128, 21, 280.0), rep(40, 32, 22), rep(20, 100, 23, 150.0, True), rep(33, 128, 24, 330.0, True)]
    slots = [add(b, r, 30, integrator=integ) for r in reps]
    b.run(18)
    b.run(12)
    est = b.estimators()
    for s, r in zip(slots, reps):
        c = orc.Sim(r["x0"], r["mass"], T=r["T"], dt=r["dt"], potential=1, ff=r["ff"], box=r["box"],
                    seed=r["seed"], integrator=integ)
        c.run(30)
        x, v, st = b.get_state(s)
        assert st == 30
        assert_split_close(x, v, est[s], c, c.estimators(), "P = %d" % r["x0"].shape[0])
    solo = pimd.Batch(1)
    t = add(solo, reps[0], 30, integrator=integ)
    solo.run(18)
    solo.run(12)
    xs, vs, _ = solo.get_state(t)
    xb, vb, _ = b.get_state(slots[0])
    assert np.array_equal(xs, xb) and np.array_equal(vs, vb)
    b.close()


def test_batch_ffma_transforms_agree_with_oracle(orc, pimd):
    """The comparison path of the transforms (every replica on the block-item
    kernel with FP32 FMA transforms) computes the same split-precision step:
    against the oracle at the split bars, bead counts 8, 32, 64 and 128."""
    b = pimd.Batch(4)
    b.set_transforms("ffma")
    reps = [MIX[0], MIX[2], MIX[3], rep(20, 128, 25)]
    slots = [add(b, r, 30) for r in reps]
    b.run(30)
    est = b.estimators()
    for s, r in zip(slots, reps):
        c = orc.Sim(r["x0"], r["mass"], T=r["T"], dt=r["dt"], potential=1, ff=r["ff"], box=r["box"],
                    seed=r["seed"])
        c.run(30)
        x, v, st = b.get_state(s)
        assert st == 30
        assert_split_close(x, v, est[s], c, c.estimators(), "FFMA P = %d" % r["x0"].shape[0])
    b.close()
