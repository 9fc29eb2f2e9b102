"""Pins for oracle/philox.py.

* The word stream: compared bit for bit with an independent implementation of
  Philox-4x32-10 that ships in the image, Triton's `tl.philox` (its own
  source, run on the CPU by Triton's interpreter in a child process).  That
  implementation fixes the multipliers, the Weyl key increments, the round
  structure and the 10 rounds of Salmon et al. (SC'11), and the split of a
  64-bit seed into the key (low word, high word).
* The counter layout and the transforms: prefix stability, seeds and streams
  that differ, statistical properties of the words, the Gaussians and the
  Rademacher signs.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import scipy.stats as st

from oracle import philox

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Child program: Triton's tl.philox on given counters and a 64-bit seed, in the
# interpreter (TRITON_INTERPRET=1 must be set before triton is imported).
_TRITON_CHILD = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np
import torch
import triton
import triton.language as tl

@triton.jit
def _k(c_ptr, out_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4 * i + 0)
    c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2)
    c3 = tl.load(c_ptr + 4 * i + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a)
    tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c)
    tl.store(out_ptr + 4 * i + 3, d)

req = json.load(sys.stdin)
res = []
for case in req:
    c = np.array(case["counters"], dtype=np.uint32).reshape(-1, 4)
    n = c.shape[0]
    ct = torch.from_numpy(c.view(np.int32).copy())
    out = torch.empty_like(ct)
    _k[(1,)](ct, out, case["seed"], N=n)
    res.append(out.numpy().view(np.uint32).reshape(-1).tolist())
json.dump(res, sys.stdout)
"""


def _triton_philox(cases):
    pytest.importorskip("triton")
    env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", _TRITON_CHILD], input=json.dumps(cases), capture_output=True,
                       text=True, env=env, timeout=600)
    if r.returncode != 0:
        pytest.skip("Triton interpreter unavailable: %s" % r.stderr.strip().splitlines()[-1:])
    return [np.array(v, dtype=np.uint32).reshape(-1, 4) for v in json.loads(r.stdout)]


def test_word_stream_equals_triton_philox4x32_10():
    rng = np.random.default_rng(2024)
    cases = []
    # edge counters and keys (all zero, all ones, one word set) plus random ones;
    # the number of counters per case is a power of two (tl.arange)
    edge = np.array([[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 0, 0, 0x80000000],
                     [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]], dtype=np.uint64)
    ctr = np.concatenate([edge, rng.integers(0, 2 ** 32, size=(64 - len(edge), 4), dtype=np.uint64)])
    for seed in (0, 0xFFFFFFFFFFFFFFFF, 1, 1 << 32, 0xA4093822299F31D0, 12345):
        cases.append({"seed": seed, "counters": ctr.astype(np.uint32).reshape(-1).tolist()})
    ref = _triton_philox(cases)
    for case, want in zip(cases, ref):
        c = np.array(case["counters"], dtype=np.uint32).reshape(-1, 4)
        k0, k1 = case["seed"] & 0xFFFFFFFF, case["seed"] >> 32
        got = np.stack(philox.philox4x32_10(c[:, 0], c[:, 1], c[:, 2], c[:, 3], k0, k1), axis=-1)
        np.testing.assert_array_equal(got, want)


def test_gaussian_and_rademacher_counters_equal_triton():
    # the streams' counter layout on top of the pinned block function: words of
    # vector s, group g are Philox((g, s, 0, 0)) for z and ((g, s, 1, 0)) for probes
    seed = 0x0123456789ABCDEF
    ng, nv = 8, 4
    g = np.tile(np.arange(ng), nv)
    s = np.repeat(np.arange(nv), ng)
    cz = np.stack([g, s, np.zeros_like(g), np.zeros_like(g)], -1).astype(np.uint32)
    cr = np.stack([g, s, np.ones_like(g), np.zeros_like(g)], -1).astype(np.uint32)
    tz, tr = _triton_philox([{"seed": seed, "counters": cz.reshape(-1).tolist()},
                             {"seed": seed, "counters": cr.reshape(-1).tolist()}])
    np.testing.assert_array_equal(philox.gaussian_words(nv, 4 * ng, seed), tz.reshape(nv, 4 * ng))
    bits = (tr.reshape(nv, 4 * ng)[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1
    want = np.where(bits.reshape(nv, -1) == 1, 1.0, -1.0)
    np.testing.assert_array_equal(philox.rademacher(nv, 128 * ng, seed), want)


def test_counter_layout_is_prefix_stable():
    a = philox.gaussian(3, 1000, seed=12345)
    b = philox.gaussian(5, 1003, seed=12345)
    np.testing.assert_array_equal(a, b[:3, :1000])
    r1 = philox.rademacher(2, 300, seed=9)
    r2 = philox.rademacher(4, 1000, seed=9)
    np.testing.assert_array_equal(r1, r2[:2, :300])


def test_seeds_and_streams_differ():
    a = philox.gaussian_words(1, 4096, seed=1)
    b = philox.gaussian_words(1, 4096, seed=2)
    c = philox.gaussian_words(1, 4096, seed=1 + (1 << 32))
    assert np.mean(a == b) < 0.01 and np.mean(a == c) < 0.01


def test_word_uniformity():
    w = philox.gaussian_words(4, 1 << 16, seed=77).reshape(-1)
    # top byte histogram: chi-square against uniform
    hist = np.bincount((w >> 24).astype(np.int64), minlength=256)
    chi2 = st.chisquare(hist)
    assert chi2.pvalue > 1e-4
    # every bit is set about half the time
    bits = np.array([(w >> b) & 1 for b in range(32)]).mean(axis=1)
    assert np.all(np.abs(bits - 0.5) < 0.01)


def test_gaussian_moments_and_ks():
    z = philox.gaussian(8, 1 << 15, seed=3).reshape(-1)
    assert abs(z.mean()) < 5 / np.sqrt(len(z))
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / len(z))
    assert st.kstest(z, "norm").pvalue > 1e-4
    # neighbouring elements and neighbouring vectors are uncorrelated
    Z = philox.gaussian(2, 1 << 16, seed=3)
    assert abs(np.corrcoef(Z[0], Z[1])[0, 1]) < 5 / np.sqrt(Z.shape[1])
    assert abs(np.corrcoef(Z[0][:-1], Z[0][1:])[0, 1]) < 5 / np.sqrt(Z.shape[1])


def test_rademacher_balance():
    r = philox.rademacher(16, 1 << 14, seed=5)
    assert set(np.unique(r)) == {-1.0, 1.0}
    assert abs(r.mean()) < 5 / np.sqrt(r.size)
