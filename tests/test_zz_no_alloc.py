"""sph_sort_keys_static: the cell-key radix sort for callers that cannot allocate
device memory (their memory belongs to another framework's pool, or they must not
allocate mid-step).  It sorts with a fixed static device buffer only; its output
must equal, bit for bit, the sorted keys and permutation that sph_build_cells
produces for the same particles.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1508_00115_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _build_sorted(d):
    """Sorted keys, permutation and grid size from the existing entry point."""
    n = d["x"].size
    ctx = binding.Context(n)
    parts = binding.Particles(d)
    ctx.build_cells(parts)
    keys = ctx.cell_keys().view(np.uint32).copy()
    perm = ctx.permutation()
    nc = ctx.stats()["nc"]
    ctx.close()
    return keys, perm, nc


def _static_sort(keys: np.ndarray, bits: int):
    n = keys.size
    kin = torch.as_tensor(keys.view(np.int32).copy()).cuda()
    kout = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    pout = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = binding.lib().sph_sort_keys_static(ctypes.c_void_p(kin.data_ptr()),
                                            ctypes.c_void_p(kout.data_ptr()),
                                            ctypes.c_void_p(pout.data_ptr()), n, bits,
                                            ctypes.c_void_p(stream))
    assert rc == binding.SPH_OK
    torch.cuda.synchronize()
    return kout.cpu().numpy().view(np.uint32), pout.cpu().numpy().view(np.uint32)


def test_static_sort_matches_build_on_two_calls_in_a_row():
    for seed in (21, 22):
        d = inputs.uniform(60000, seed=seed)
        ks, perm, nc = _build_sorted(d)
        # unsorted build keys of the input order: cell * 8 + octant of the wrapped
        # position inside its cell (bits x, y, z at or above the cell centre)
        pos = [oracle.wrap(d[k], 1.0) for k in ("x", "y", "z")]
        cell = oracle.cell_keys(*pos, 1.0, nc).astype(np.uint32)
        L = 1.0 / nc
        idx = (cell % nc, (cell // nc) % nc, cell // (nc * nc))
        octant = sum(((p >= (i + 0.5) * L).astype(np.uint32) << b)
                     for b, (p, i) in enumerate(zip(pos, idx)))
        keys = (cell << 3) | octant
        bits = int(nc ** 3 - 1).bit_length() + 3
        ko, po = _static_sort(keys, bits)
        assert np.array_equal(ko >> 3, ks)
        assert np.array_equal(po.astype(np.int64), perm)


@pytest.mark.parametrize("bits", [8, 13, 16, 24, 32])
def test_static_sort_random_keys_match_stable_argsort(bits):
    """Random keys, every pass count (1-4 passes: an odd count writes the outputs in
    the first pass straight from the input), keys with stray bits above key_bits
    (they must take no part in the order), two calls in a row."""
    rng = np.random.default_rng(100 + bits)
    mask = np.uint32((1 << bits) - 1)
    for n in (1, 4095, 4097, 50001):
        keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
        # half the keys take few distinct low values, so that stability decides many
        # slots; their high bits stay random
        half = n // 2
        keys[:half] = (keys[:half] & ~mask) | ((keys[:half] & mask) % np.uint32(7))
        low = keys & mask
        want = np.argsort(low, kind="stable")
        for _ in range(2):
            ko, po = _static_sort(keys, bits)
            assert np.array_equal(po.astype(np.int64), want)
            assert np.array_equal(ko, keys[want])


def test_static_sort_at_the_size_limit():
    n = binding.SPH_SORT_STATIC_MAX_N
    rng = np.random.default_rng(7)
    keys = rng.integers(0, 1 << 20, n, dtype=np.uint32)
    want = np.argsort(keys, kind="stable")
    for bits in (20, 24):
        ko, po = _static_sort(keys, bits)
        assert np.array_equal(po.astype(np.int64), want)
        assert np.array_equal(ko, keys[want])


def test_static_sort_rejects_oversize_without_gpu_work():
    L = binding.lib()
    rc = L.sph_sort_keys_static(None, None, None, binding.SPH_SORT_STATIC_MAX_N + 1, 16, None)
    assert rc == binding.SPH_ERR_INVALID_ARG
    rc = L.sph_sort_keys_static(None, None, None, 10, 0, None)
    assert rc == binding.SPH_ERR_INVALID_ARG
