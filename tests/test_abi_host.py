"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every symbol include/blockcg.h declares, and validates arguments."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1710_09745_gb300 import build, binding
    build.build()
    return binding.load_library()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "blockcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(blockcg_[a-zA-Z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_1710_09745_gb300 import binding
    names = declared_symbols()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.ABI_SYMBOLS) == names


def test_default_params_and_status_strings(lib):
    from paper_1710_09745_gb300.binding import Params
    p = Params()
    lib.blockcg_default_params(ct.byref(p))
    assert p.max_iter == 100000 and abs(p.ru_delta - 0.1) < 1e-15 and p.prec == 0
    for s in range(8):
        assert lib.blockcg_status_string(s)


@pytest.mark.parametrize("dims,ok", [((4, 4, 4, 4), True), ((3, 4, 4, 4), False),
                                     ((4, 4, 0, 4), False), ((2, 2, 2, 2), True),
                                     ((4, 4, 4, 5), False)])
def test_create_validates_dims(lib, dims, ok):
    h = ct.c_void_p()
    d = (ct.c_int * 4)(*dims)
    rc = lib.blockcg_create(ct.byref(h), d, 0.1, None, None)
    assert (rc == 0) == ok
    if ok:
        lib.blockcg_destroy(h)


def test_create_rejects_bad_mass_and_params(lib):
    from paper_1710_09745_gb300.binding import Params
    h = ct.c_void_p()
    d = (ct.c_int * 4)(4, 4, 4, 4)
    assert lib.blockcg_create(ct.byref(h), d, float("nan"), None, None) == 1
    p = Params()
    lib.blockcg_default_params(ct.byref(p))
    p.ru_delta = 1.5
    assert lib.blockcg_create(ct.byref(h), d, 0.1, ct.byref(p), None) == 1
    p.ru_delta = 0.1
    p.prec = 7
    assert lib.blockcg_create(ct.byref(h), d, 0.1, ct.byref(p), None) == 1


def test_sizes_and_unready_handle(lib):
    from paper_1710_09745_gb300.binding import Params
    h = ct.c_void_p()
    d = (ct.c_int * 4)(8, 8, 8, 8)
    assert lib.blockcg_create(ct.byref(h), d, 0.1, None, None) == 0
    Vh = 8 ** 4 // 2
    # double-float links: 2 parities x 16 hops x 9 entries x 16 bytes
    assert lib.blockcg_gauge_bytes(h) >= 2 * 16 * 9 * Vh * 16
    w1 = lib.blockcg_workspace_bytes(h, 1)
    w16 = lib.blockcg_workspace_bytes(h, 16)
    assert 0 < w1 < w16
    assert lib.blockcg_workspace_bytes(h, 0) == 0 and lib.blockcg_workspace_bytes(h, 65) == 0
    # no gauge / workspace yet: refused without touching the GPU
    assert lib.blockcg_apply_MdagM(h, ct.c_void_p(16), ct.c_void_p(16), 1) == 3
    assert lib.blockcg_solve(h, ct.c_void_p(16), ct.c_void_p(16), 1, 1e-10, None) == 3
    assert lib.blockcg_set_workspace(h, None, 0) == 3
    assert lib.blockcg_load_gauge(h, None, None, None, 0) == 1
    assert lib.blockcg_last_error(h)
    lib.blockcg_destroy(h)
    p = Params()
    lib.blockcg_default_params(ct.byref(p))
    p.prec = 2
    assert lib.blockcg_create(ct.byref(h), d, 0.1, ct.byref(p), None) == 0
    # mixed form keeps a second (FP32) copy of the links
    assert lib.blockcg_gauge_bytes(h) >= 2 * 16 * 9 * Vh * (16 + 8)
    lib.blockcg_destroy(h)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1710_09745_gb300 import binding
    with pytest.raises(RuntimeError):
        binding._lib = None
        try:
            binding.load_library(str(tmp_path / "missing.so"))
        finally:
            binding._lib = None


def test_batch_entry_points_validate_without_gpu(lib):
    """Argument checks of the batch entry points run before any CUDA call."""
    b = ct.c_void_p()
    assert lib.blockcg_batch_create(ct.byref(b), None, 1, None) == 1
    hs = (ct.c_void_p * 2)(None, None)
    assert lib.blockcg_batch_create(ct.byref(b), hs, 0, None) == 1
    assert lib.blockcg_batch_create(ct.byref(b), hs, 2, None) == 1  # null handles
    assert lib.blockcg_batch_create(None, hs, 2, None) == 1
    assert lib.blockcg_batch_solve(None, None, None, None, 1e-10, 1, None, None, None) == 1
    lib.blockcg_batch_destroy(None)
    assert lib.blockcg_batch_last_error(None) == b"null batch"


def test_batch_rejects_repeated_handles(lib):
    """Two entries with the same handle would share one workspace."""
    h = ct.c_void_p()
    d = (ct.c_int * 4)(4, 4, 4, 4)
    assert lib.blockcg_create(ct.byref(h), d, 0.1, None, None) == 0
    try:
        hs = (ct.c_void_p * 2)(h, h)
        b = ct.c_void_p()
        assert lib.blockcg_batch_create(ct.byref(b), hs, 2, None) == 1
    finally:
        lib.blockcg_destroy(h)


def test_link_grad_validates_without_gpu(lib):
    h = ct.c_void_p()
    d = (ct.c_int * 4)(4, 4, 4, 4)
    assert lib.blockcg_link_grad(None, None, None, 1, None, None) == 1
    assert lib.blockcg_create(ct.byref(h), d, 0.1, None, None) == 0
    try:
        # no gauge field and no workspace yet: refused before any device work
        assert lib.blockcg_link_grad(h, None, None, 1, None, None) != 0
        assert lib.blockcg_link_grad(h, None, None, 0, None, None) == 1
    finally:
        lib.blockcg_destroy(h)


def test_link_recon_parameter_checks(lib):
    """Two-row links only with the 32- and 16-bit forms, and only 0 or 12;
    they shrink the gauge storage of those forms."""
    from paper_1710_09745_gb300.binding import Params, PREC
    d = (ct.c_int * 4)(4, 4, 4, 4)
    p = Params()
    lib.blockcg_default_params(ct.byref(p))
    assert p.link_recon == 0
    sizes = {}
    for prec, recon, ok in (("f64", 12, False), ("f64_native", 12, False), ("mixed_f32", 7, False),
                            ("mixed_f32", 12, True), ("mixed_f16", 12, True),
                            ("mixed_bf16", 12, True), ("mixed_f32", 0, True)):
        lib.blockcg_default_params(ct.byref(p))
        p.prec, p.link_recon = PREC[prec], recon
        h = ct.c_void_p()
        rc = lib.blockcg_create(ct.byref(h), d, 0.1, ct.byref(p), None)
        assert (rc == 0) == ok, (prec, recon)
        if ok:
            sizes[(prec, recon)] = lib.blockcg_gauge_bytes(h)
            lib.blockcg_destroy(h)
    V = 256
    fine = 2 * (V // 2 // 32) * 16 * 9 * 32 * 16          # FP64 links, both parities
    f32_full = 2 * (V // 2 // 32) * 16 * 9 * 32 * 8
    f32_two = 2 * (V // 2 // 32) * 16 * 6 * 32 * 8
    # the mixed forms also keep double-float links for their reliable updates
    # (16 bytes per complex entry, the size of the FP64 copy)
    ru_df = fine
    assert sizes[("mixed_f32", 0)] == fine + f32_full + ru_df
    assert sizes[("mixed_f32", 12)] == fine + f32_two + ru_df + 256


def _c_layout(struct, fields):
    """offsetof/sizeof of a struct of include/blockcg.h, from a C program
    compiled against the header (gcc, host only)."""
    import subprocess
    import tempfile
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "blockcg.h"', "int main(void) {",
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return [int(v) for v in out]


@pytest.mark.parametrize("struct,cls", [("blockcg_params", "Params"), ("blockcg_stats", "Stats"),
                                        ("blockcg_batch_stats", "BatchStats"),
                                        ("blockcg_many_stats", "ManyStats")])
def test_binding_structs_match_the_header_layout(struct, cls):
    """The ctypes mirrors of the ABI structs have the C compiler's field
    offsets and sizes, including the per-right-hand-side residual pointer of
    blockcg_stats and the wait limit of blockcg_params."""
    from paper_1710_09745_gb300 import binding
    C = getattr(binding, cls)
    names = [f[0] for f in C._fields_]
    got = _c_layout(struct, names)
    assert got[0] == ct.sizeof(C)
    for name, off in zip(names, got[1:]):
        assert getattr(C, name).offset == off, name
    if struct == "blockcg_stats":
        assert "true_rel_res" in names
    if struct == "blockcg_params":
        assert "wait_limit_ns" in names


def test_wait_limit_must_not_be_negative(lib):
    from paper_1710_09745_gb300.binding import Params
    h = ct.c_void_p()
    d = (ct.c_int * 4)(4, 4, 4, 4)
    p = Params()
    lib.blockcg_default_params(ct.byref(p))
    assert p.wait_limit_ns == 0
    p.wait_limit_ns = -1
    assert lib.blockcg_create(ct.byref(h), d, 0.1, ct.byref(p), None) == 1
    p.wait_limit_ns = 1000
    assert lib.blockcg_create(ct.byref(h), d, 0.1, ct.byref(p), None) == 0
    lib.blockcg_destroy(h)


def test_dslash_variant_encoding(lib):
    """R in {1, 2, 4, 8} plus at most the documented kernel flags."""
    from paper_1710_09745_gb300.binding import Params
    d = (ct.c_int * 4)(4, 4, 4, 4)
    for v, want in [(4, 0), (256 + 4, 0), (512 + 2, 0), (4096 + 8, 0), (8192 + 2, 0),
                    (3, 1), (2048 + 256 + 4, 1), (16384 + 4, 1), (4096, 1), (8192, 1)]:
        h = ct.c_void_p()
        p = Params()
        lib.blockcg_default_params(ct.byref(p))
        p.dslash_variant = v
        assert lib.blockcg_create(ct.byref(h), d, 0.1, ct.byref(p), None) == want, v
        if want == 0:
            lib.blockcg_destroy(h)


def test_solve_many_validates_without_gpu(lib):
    h = ct.c_void_p()
    d = (ct.c_int * 4)(4, 4, 4, 4)
    assert lib.blockcg_solve_many(None, None, None, 1, 1e-10, 0, None) == 1
    assert lib.blockcg_set_tune_cache(None, b"x") == 1
    assert lib.blockcg_create(ct.byref(h), d, 0.1, None, None) == 0
    try:
        p = ct.c_void_p(16)
        assert lib.blockcg_solve_many(h, p, p, 0, 1e-10, 0, None) == 1      # m_rhs < 1
        assert lib.blockcg_solve_many(h, p, p, 4, 1e-10, 65, None) == 1     # width > 64
        assert lib.blockcg_solve_many(h, p, p, 4, -1.0, 0, None) == 1       # tol
        assert lib.blockcg_solve_many(h, p, p, 4, 1e-10, 0, None) == 3      # no workspace
        assert lib.blockcg_set_tune_cache(h, None) == 0
    finally:
        lib.blockcg_destroy(h)
