"""C ABI: the library loads, exports every entry point declared in include/spiir.h, and rejects
invalid arguments on the host before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2011_06787_b300 as sp
from paper_2011_06787_b300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(spiir_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    L = native.lib()
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(native.SIGNATURES), declared ^ set(native.SIGNATURES)


def test_version_and_error_text():
    assert sp.version() >= 100
    assert isinstance(native.last_error(), str)


@pytest.mark.parametrize("kwargs,msg", [
    (dict(n_det=0), "n_det"),
    (dict(offsets=[0, 3, 2]), "decrease"),
    (dict(offsets=[1, 2, 3]), "filter_offsets[0]"),
    (dict(a1=np.array([0.5, 1.2, 0.3], dtype=np.complex64)), "|a1| >= 1"),
    (dict(b0=np.array([np.nan, 0, 0], dtype=np.complex64)), "non-finite"),
    (dict(delay=[0, -1, 2]), "delay"),
])
def test_bank_create_rejects_invalid_arguments(kwargs, msg):
    args = dict(n_det=2, offsets=[0, 1, 3], a1=np.full(3, 0.5, np.complex64), b0=np.ones(3, np.complex64),
                delay=[0, 1, 2])
    args.update(kwargs)
    with pytest.raises(sp.SpiirError) as e:
        sp.Bank(args["n_det"], args["offsets"], args["a1"], args["b0"], args["delay"])
    assert e.value.code == native.EINVAL
    assert msg in str(e.value)


def test_sky_create_rejects_invalid_arguments():
    with pytest.raises(sp.SpiirError):
        sp.Sky(np.zeros((4, 5), np.int32), np.zeros((4, 5, 2), np.float32), np.zeros((4, 5, 3), np.float32))
    with pytest.raises(sp.SpiirError):
        sp.Sky(np.full((4, 3), 5000, np.int32), np.zeros((4, 3, 2), np.float32), np.zeros((4, 3, 1), np.float32))


def test_sky_tables_rejects_bad_geometry():
    pos = np.zeros((3, 3))
    arms = np.eye(3)
    with pytest.raises(sp.SpiirError):
        sp.sky_tables(pos, arms * 2.0, arms, np.ones(3), 4, 2048.0)   # arms not unit
    with pytest.raises(sp.SpiirError):
        sp.sky_tables(pos, arms, arms, np.array([1.0, -1.0, 1.0]), 4, 2048.0)  # negative sigma
    with pytest.raises(sp.SpiirError):
        sp.sky_tables(pos, arms, arms, np.ones(3), 0, 2048.0)


def test_batch_create_rejects_invalid_arguments():
    import synth
    banks = synth.multirate_banks(n_banks=2, t_range=(2, 4), f_range=(5, 10), seed_sub=9)

    class FakeSky:  # any handle; validation of the band layout happens before the sky is used
        handle = None

    for factors, chunk, msg in (((1, 3, 16), 512, "power of two"), ((1, 4, 16), 520, "multiple"),
                                ((1, 4, 16), 16, "multiple"), ((1, 4, 16), 512, "sky is NULL")):
        with pytest.raises(sp.SpiirError) as e:
            sp.Batch(3, banks, factors, FakeSky(), chunk)
        assert e.value.code == native.EINVAL and msg in str(e.value)
    bad = [(o, a, b, d, np.full_like(bb, 3)) for o, a, b, d, bb in banks]
    with pytest.raises(sp.SpiirError) as e:
        sp.Batch(3, bad, (1, 4, 16), FakeSky(), 512)
    assert "band 3" in str(e.value)


def test_wait_timeout_hook_rejects_bad_limits():
    L = native.lib()
    for it in (0, (1 << 26) + 1):
        assert L.spiir_debug_wait_timeout(it, None) == native.EINVAL


def test_select_workspace_size():
    """One 64-bit slot per (detector, template, second), one 64-bit key per (detector, sample)
    and one word for the compaction's block counter; invalid sizes are rejected."""
    L = native.lib()
    nb = ctypes.c_size_t()
    for T, nd, n, ps in [(1024, 3, 2048, 2048), (37, 3, 5000, 2048), (1, 1, 1, 7)]:
        assert L.spiir_select_workspace_bytes(T, nd, n, ps, ctypes.byref(nb)) == 0
        n_sec = -(-n // ps)
        assert nb.value == 8 * (nd * (T * n_sec + n) + 1)
    assert L.spiir_select_workspace_bytes(0, 3, 2048, 2048, ctypes.byref(nb)) == native.EINVAL
    assert L.spiir_select_workspace_bytes(16, 3, 0, 2048, ctypes.byref(nb)) == native.EINVAL


def test_header_compiles_as_plain_c(tmp_path):
    """include/spiir.h is a C header: it compiles as C99 with warnings as errors (no C++ or CUDA
    types in the signatures)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "spiir.h"\nint main(void) { return SPIIR_OK; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I",
                        os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
