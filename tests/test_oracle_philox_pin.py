"""Pin of the oracle's Philox4x32-10 against an implementation it shares
nothing with: the Philox of the triton library (triton.language.random,
written from Salmon, Moraes, Dror & Shaw, SC'11), run on the CPU through
triton's interpreter.  A wrong multiplier, Weyl constant, word order or
high/low half in the oracle fails here; statistics and avalanche tests
alone would not see it.

The library's generator runs in a child process, because its interpreter is
switched on by an environment variable read when kernels are defined."""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle

pytest.importorskip("triton")

_CHILD = textwrap.dedent(
    """
    import json, os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def rounds(c_ptr, k_ptr, out_ptr, N: tl.constexpr):
        i = tl.arange(0, N)
        c0 = tl.load(c_ptr + 4 * i + 0)
        c1 = tl.load(c_ptr + 4 * i + 1)
        c2 = tl.load(c_ptr + 4 * i + 2)
        c3 = tl.load(c_ptr + 4 * i + 3)
        k0 = tl.load(k_ptr + 2 * i + 0)
        k1 = tl.load(k_ptr + 2 * i + 1)
        r0, r1, r2, r3 = tl.random.philox_impl(c0, c1, c2, c3, k0, k1, 10)
        tl.store(out_ptr + 4 * i + 0, r0)
        tl.store(out_ptr + 4 * i + 1, r1)
        tl.store(out_ptr + 4 * i + 2, r2)
        tl.store(out_ptr + 4 * i + 3, r3)

    req = json.loads(sys.stdin.read())
    ctr = np.array(req["ctr"], dtype=np.uint64).astype(np.uint32)
    key = np.array(req["key"], dtype=np.uint64).astype(np.uint32)
    n = len(ctr) // 4
    c = torch.from_numpy(ctr.copy())
    k = torch.from_numpy(key.copy())
    out = torch.zeros_like(c)
    rounds[(1,)](c, k, out, N=n)
    print(json.dumps([int(v) for v in out.numpy()]))
    """
)


def _library_philox(keys: np.ndarray, ctrs: np.ndarray) -> np.ndarray:
    """Philox4x32-10 of the triton library for each (key, counter) row."""
    n = len(keys)
    assert n & (n - 1) == 0, "the interpreted kernel takes a power-of-two block"
    req = {"ctr": [int(v) for v in ctrs.ravel()], "key": [int(v) for v in keys.ravel()]}
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _CHILD], input=json.dumps(req), capture_output=True,
                       text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.array(json.loads(r.stdout.strip().splitlines()[-1]), dtype=np.uint64).astype(np.uint32).reshape(n, 4)


def _cases() -> tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng(20131021)
    n = 256
    keys = rng.integers(0, 2**32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctrs = rng.integers(0, 2**32, (n, 4), dtype=np.uint64).astype(np.uint32)
    # edge words: all zero, all ones, single bits, and the counter layout the
    # method uses (id, step low, step high, species<<24 | tag<<16 | sub)
    keys[0], ctrs[0] = 0, 0
    keys[1], ctrs[1] = 0xFFFFFFFF, 0xFFFFFFFF
    keys[2], ctrs[2] = (1, 0), (1, 0, 0, 0)
    keys[3], ctrs[3] = (0, 1), (0, 0, 0, 0x80000000)
    keys[4], ctrs[4] = (1, 0), (12345, 400, 0, (1 << 24) | (2 << 16) | 1)
    keys[5], ctrs[5] = (2, 0), (2047999, 3999, 0, (2 << 16))
    return keys, ctrs


def test_oracle_philox_equals_library_philox():
    keys, ctrs = _cases()
    ref = _library_philox(keys, ctrs)
    got = np.stack([oracle.philox(k, c) for k, c in zip(keys, ctrs)])
    bad = np.nonzero(np.any(got != ref, axis=1))[0]
    assert bad.size == 0, "first mismatch at row %d: key %s ctr %s oracle %s library %s" % (
        bad[0], keys[bad[0]], ctrs[bad[0]], got[bad[0]], ref[bad[0]])


def test_oracle_philox_stream_equals_library_philox():
    # the stream form the oracle's sampling uses: counter word 0 runs
    key = np.array([0xDEADBEEF, 7], dtype=np.uint32)
    n = 128
    ctrs = np.zeros((n, 4), dtype=np.uint32)
    ctrs[:, 0] = np.arange(n, dtype=np.uint32) + np.uint32(0xFFFFFFC0)  # wraps past 2^32
    ctrs[:, 1], ctrs[:, 2], ctrs[:, 3] = 5, 0, 3 << 16
    ref = _library_philox(np.tile(key, (n, 1)), ctrs)
    got = oracle.philox_stream(key, (0xFFFFFFC0, 5, 0, 3 << 16), n)
    assert np.array_equal(got, ref)
