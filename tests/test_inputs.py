"""The seeded input generators (paper_2406_09857_gb300/synth.py) against their published
definitions, so that every machine draws the same integers:

- SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) against a plain-integer restatement and its
  well-known first output for seed 0 (0xE220A8397B1DCDAF);
- integers in a range by rejection: in range, every value reached, deterministic per seed;
- uniforms in [0, 1) are the top 53 bits of the outputs (exact);
- Kostlan scales are square roots of exact multinomials;
- the benchmark's curve is the documented size (two polynomials of C(103, 3) terms).
The N(0,1) draws go through the platform's log and cos: they are checked for their law here,
not for their last bits.
"""
import math

import numpy as np

from paper_2406_09857_gb300 import synth

M64 = (1 << 64) - 1


def _splitmix64(seed, n):
    s, out = seed, []
    for _ in range(n):
        s = (s + 0x9E3779B97F4A7C15) & M64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_definition():
    assert int(synth.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF
    for seed in (0, 1, synth.BASE_SEED, M64):
        assert [int(x) for x in synth.splitmix64(seed, 50)] == _splitmix64(seed, 50)
    # a stream continues where it stopped
    st = synth.Stream(12345)
    a, b = st.raw(7), st.raw(9)
    assert [int(x) for x in np.concatenate([a, b])] == _splitmix64(12345, 16)


def test_uniform_int_and_unit():
    v = synth.Stream(7).uniform_int(-3, 5, 5000)
    assert v.min() == -3 and v.max() == 5 and set(v.tolist()) == set(range(-3, 6))
    assert np.array_equal(v, synth.Stream(7).uniform_int(-3, 5, 5000))
    u = synth.Stream(8).unit(1000)
    raw = _splitmix64(8, 1000)
    assert np.array_equal(u, np.array([(x >> 11) * 2.0 ** -53 for x in raw]))
    assert (u >= 0).all() and (u < 1).all()


def test_normal_law():
    z = synth.Stream(9).normal(200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    assert abs((np.abs(z) < 1).mean() - 0.6827) < 0.005


def test_kostlan_scale_exact():
    e = synth.dense_total_degree(3, 12)
    sc = synth.kostlan_scale(e, 12)
    for a, s in zip(e.tolist()[::37], sc.tolist()[::37]):
        m = math.factorial(12) // (math.factorial(12 - sum(a)) *
                                   math.prod(math.factorial(x) for x in a))
        assert s == math.sqrt(float(m))


def test_curve_workload_size():
    s = synth.curve()
    assert s.k == 3 and len(s.polys) == 2 and s.depth == 10
    for e, c in s.polys:
        assert e.shape == (math.comb(103, 3), 3) and c.shape == (math.comb(103, 3),)
        assert (e.sum(axis=1) <= 100).all()
