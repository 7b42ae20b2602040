"""Host-side checks of the C-ABI library (no GPU needed, no compute calls):
the library builds for sm_103a, loads, exports every entry point include/sph.h
declares, and its structs have the layout the Python binding assumes."""
import ctypes
import os
import pathlib
import subprocess

import pytest

from paper_1508_00115_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return binding.lib()


def test_library_exports_every_declared_symbol(L):
    names = binding.header_symbols()
    assert {"sph_init", "sph_build_cells", "sph_density", "sph_force", "sph_step"} <= set(names)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_struct_layout_matches_header():
    """Compile a probe against include/sph.h with gcc and compare sizeof/offsetof
    with the ctypes mirrors."""
    scratch = pathlib.Path(ROOT) / "tests" / "_build"  # git-ignored
    scratch.mkdir(exist_ok=True)
    src = scratch / "probe.c"
    fields = {
        "sph_params": [f for f, _ in binding.sph_params._fields_],
        "sph_particles": [f for f, _ in binding.sph_particles._fields_],
        "sph_conserved": [f for f, _ in binding.sph_conserved._fields_],
        "sph_stats": [f for f, _ in binding.sph_stats._fields_],
        "sph_bin_stats": [f for f, _ in binding.sph_bin_stats._fields_],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sph.h"', "int main(void){"]
    for s, fs in fields.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fs:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = scratch / "probe"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    out = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).split("\n")
               if l)
    for s in fields:
        cls = getattr(binding, s)
        assert int(out[s]) == ctypes.sizeof(cls), s
        for f in fields[s]:
            assert int(out[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)


def test_constants_match_header():
    """Every SPH_* constant the binding mirrors (macros and enumerators) has the
    header's value."""
    names = [k for k in dir(binding) if k.startswith("SPH_") and isinstance(getattr(binding, k), int)]
    scratch = pathlib.Path(ROOT) / "tests" / "_build"  # git-ignored
    scratch.mkdir(exist_ok=True)
    src = scratch / "consts.c"
    lines = ['#include <stdio.h>', '#include "sph.h"', "int main(void){"]
    for k in names:
        lines.append(f'printf("{k} %lld\\n", (long long)({k}));')  # (a name the header lacks fails to compile)
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = scratch / "consts"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).split("\n") if l)
    assert sorted(out) == sorted(names)
    for k, v in out.items():
        assert int(v) == getattr(binding, k), k


def test_default_params(L):
    p = binding.sph_default_params()
    assert p.n_ngb == 48.0 and abs(p.gamma - 5 / 3) < 1e-7 and p.kernel == 0
    assert p.max_h_iter == 30 and p.use_balsara == 1 and p.box_size == 1.0


def test_init_rejects_bad_params_without_touching_the_device(L):
    for k, v in (("n", -1), ("box_size", 0.0), ("gamma", 1.0), ("n_ngb", 5.0), ("h_tol", 0.0),
                 ("cell_factor", 0.5), ("max_h_iter", 0), ("kernel", 3), ("cfl", 0.0),
                 ("tile_width", 24)):
        p = binding.sph_default_params()
        setattr(p, k, v)
        h = ctypes.c_void_p(123)
        rc = L.sph_init(ctypes.byref(h), ctypes.byref(p), 0, None)
        assert rc == binding.SPH_ERR_INVALID_ARG, k
        assert not h.value


def test_null_context_is_rejected(L):
    assert L.sph_build_cells(None, None) == binding.SPH_ERR_INVALID_ARG
    assert L.sph_density(None, None, None) == binding.SPH_ERR_INVALID_ARG
    assert L.sph_force(None, None) == binding.SPH_ERR_INVALID_ARG
    assert L.sph_step(None, None, 0.0, None, None) == binding.SPH_ERR_INVALID_ARG
    assert L.sph_last_error(None) == b"null context"
    L.sph_destroy(None)


def test_oracle_and_library_share_no_code():
    """The CUDA sources never include or name the oracle, and the oracle never
    imports the package (the input generators are the one shared module)."""
    csrc = os.path.join(ROOT, "paper_1508_00115_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower() or "no oracle" in text.lower(), f
    for f in ("binding.py", "build.py"):
        text = open(os.path.join(ROOT, "paper_1508_00115_gb300", f)).read()
        assert "import oracle" not in text and "from oracle" not in text
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1508_00115_gb300" not in text.replace("paper_1508_00115_gb300/inputs.py", "")


def test_header_constants_match_binding():
    """Flags, status codes and SPH_MAX_BINS: the header's values are the binding's."""
    import re
    text = open(os.path.join(ROOT, "include", "sph.h")).read()
    defs = dict(re.findall(r"#define (SPH_\w+) (\d+)u?\b", text))
    defs.update(re.findall(r"^\s*(SPH_(?:OK|ERR_\w+)) = (\d+)", text, flags=re.M))
    assert len(defs) >= 17, defs
    for name, value in defs.items():
        if hasattr(binding, name):
            assert getattr(binding, name) == int(value), name
    assert int(defs["SPH_MAX_BINS"]) == binding.SPH_MAX_BINS


def test_static_sort_rejects_overlapping_buffers_without_gpu_work(L):
    """sph_sort_keys_static cannot sort in place: any overlap of keys_in, keys_out and
    perm_out is refused before anything touches a device (the addresses below are
    never dereferenced)."""
    n = 1000
    base = 1 << 40
    cases = [(base, base, base + 8 * n),             # keys_out == keys_in
             (base, base + 8 * n, base + 4),          # perm_out inside keys_in
             (base, base + 8 * n, base + 8 * n + 4)]  # perm_out overlaps keys_out
    for kin, kout, pout in cases:
        rc = L.sph_sort_keys_static(ctypes.c_void_p(kin), ctypes.c_void_p(kout), ctypes.c_void_p(pout), n,
                                    32, None)
        assert rc == binding.SPH_ERR_INVALID_ARG, (kin, kout, pout)
