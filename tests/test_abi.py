"""The C ABI library loads and exports every symbol include/pgs.h declares;
host-only argument checks return their status codes without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1611_00463_gb300 import build, pgs
    build.build()
    return pgs.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pgs_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["pgs_sort", "pgs_sort_copy", "pgs_workspace_bytes", "pgs_fit_splitters",
                 "pgs_fit_workspace_bytes", "pgs_get_stats", "pgs_strerror", "pgs_version"]:
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_1611_00463_gb300 import pgs
    assert sorted(pgs.EXPORTS) == declared_functions()


def test_struct_sizes_match_header(lib):
    from paper_1611_00463_gb300 import pgs
    # pgs_stats is copied byte for byte from the device block.
    assert ctypes.sizeof(pgs.pgs_stats) == 64
    assert [lib.pgs_batch_auto_partitions(n) for n in [1, 65535, 65536, 131071, 131072, 1 << 24, 1 << 30]] == \
        [1, 1, 1, 1, 2, 256, 256]
    assert ctypes.sizeof(pgs.pgs_config) == 32 + 8 * 12
    assert ctypes.sizeof(pgs.pgs_launch_record) == 24
    assert [lib.pgs_kernel_name(i).decode() for i in range(len(pgs.KERNELS))] == pgs.KERNELS


def test_strerror_and_version(lib):
    assert lib.pgs_strerror(0) == b"ok"
    assert lib.pgs_strerror(-2).startswith(b"workspace")
    assert lib.pgs_strerror(12345) == b"unknown status"
    assert re.match(rb"\d+\.\d+\.\d+", lib.pgs_version())


def test_workspace_bytes_host_only(lib):
    from paper_1611_00463_gb300 import pgs
    cfg = pgs.make_config(dtype="u64")
    small = pgs.pgs_workspace_bytes(1 << 10, 4, cfg)
    big = pgs.pgs_workspace_bytes(1 << 20, 4, cfg)
    assert 0 < small < big
    # The alternate key+payload buffer dominates: at least n * (8 + 4) bytes.
    assert big >= (1 << 20) * 12
    assert pgs.pgs_workspace_bytes(100, 0, cfg) == 0
    bad = pgs.make_config(dtype="u64")
    bad.investigator = 7
    assert pgs.pgs_workspace_bytes(100, 4, bad) == 0


def test_invalid_arguments_rejected_before_launch(lib):
    from paper_1611_00463_gb300 import pgs
    cfg = pgs.make_config()
    fake = ctypes.c_void_p(0x1000)
    # P = 0
    assert lib.pgs_sort_copy(fake, None, fake, None, 10, 0, None, ctypes.byref(cfg)) == pgs.PGS_ERR_INVALID
    # NULL keys with n > 0
    assert lib.pgs_sort_copy(None, None, None, None, 10, 2, None, ctypes.byref(cfg)) == pgs.PGS_ERR_INVALID
    # vals on one side only
    assert lib.pgs_sort_copy(fake, fake, fake, None, 10, 2, None, ctypes.byref(cfg)) == pgs.PGS_ERR_INVALID
    # n = 0 is a no-op
    assert lib.pgs_sort_copy(None, None, None, None, 0, 2, None, ctypes.byref(cfg)) == pgs.PGS_OK
    # no workspace, misaligned workspace, too small a workspace
    assert lib.pgs_sort_copy(fake, None, ctypes.c_void_p(0x2000), None, 10, 2, None,
                             ctypes.byref(cfg)) == pgs.PGS_ERR_WORKSPACE
    cfg.workspace = 0x10001
    cfg.workspace_bytes = 1 << 30
    assert lib.pgs_sort_copy(fake, None, ctypes.c_void_p(0x2000), None, 10, 2, None,
                             ctypes.byref(cfg)) == pgs.PGS_ERR_WORKSPACE
    cfg.workspace = 0x100000
    cfg.workspace_bytes = 16
    assert lib.pgs_sort_copy(fake, None, ctypes.c_void_p(0x2000), None, 10, 2, None,
                             ctypes.byref(cfg)) == pgs.PGS_ERR_WORKSPACE
    # partially overlapping input and output
    cfg.workspace_bytes = 1 << 30
    assert lib.pgs_sort_copy(ctypes.c_void_p(0x1000), None, ctypes.c_void_p(0x1004), None, 10, 2, None,
                             ctypes.byref(cfg)) == pgs.PGS_ERR_INVALID
    # bad enum values
    cfg2 = pgs.make_config()
    cfg2.dtype = 9
    assert lib.pgs_sort_copy(fake, None, fake, None, 10, 2, None, ctypes.byref(cfg2)) == pgs.PGS_ERR_INVALID
    # fit: fewer samples than partitions
    cfg3 = pgs.make_config()
    assert lib.pgs_fit_splitters(fake, 3, 8, None, ctypes.byref(cfg3), fake, None) == pgs.PGS_ERR_INVALID
    # stats: NULL
    assert lib.pgs_get_stats(None, None, None) == pgs.PGS_ERR_INVALID


def test_batch_plan_host_only(lib):
    import numpy as np
    from paper_1611_00463_gb300 import pgs
    cfg = pgs.make_config(dtype="u64")
    off = np.array([0, 10, 10, 200_000, 200_005], dtype=np.uint64)
    h = ctypes.c_void_p()
    assert lib.pgs_batch_create(off.ctypes.data, 4, None, 1, ctypes.byref(cfg), ctypes.byref(h)) == pgs.PGS_OK
    ws = lib.pgs_batch_workspace_bytes(h)
    assert ws >= 200_005 * 12
    # uploading to a misaligned or small workspace is refused before any copy
    assert lib.pgs_batch_upload(h, ctypes.c_void_p(0x1001), 1 << 40, None) == pgs.PGS_ERR_WORKSPACE
    assert lib.pgs_batch_upload(h, ctypes.c_void_p(0x1000), 16, None) == pgs.PGS_ERR_WORKSPACE
    assert lib.pgs_batch_destroy(h) == pgs.PGS_OK
    bad = np.array([0, 10, 5], dtype=np.uint64)                     # decreasing offsets
    assert lib.pgs_batch_create(bad.ctypes.data, 2, None, 1, ctypes.byref(cfg), ctypes.byref(h)) == \
        pgs.PGS_ERR_INVALID
    zeroP = np.array([0], dtype=np.uint32)
    assert lib.pgs_batch_create(off.ctypes.data, 1, zeroP.ctypes.data, 1, ctypes.byref(cfg),
                                ctypes.byref(h)) == pgs.PGS_ERR_INVALID


class _FakeDeviceTensor:
    """Stands in for a device tensor on a machine without a GPU: make_config
    reads only these attributes."""
    is_cuda = True

    def __init__(self, addr, nbytes):
        self.addr, self.nbytes = addr, nbytes

    def is_contiguous(self):
        return True

    def data_ptr(self):
        return self.addr

    def numel(self):
        return self.nbytes

    def element_size(self):
        return 1


def test_config_keeps_its_tensors_alive():
    """A config holds raw addresses; it must also hold the tensors, or a
    workspace built inline is freed (and its memory reused) while the library
    still writes into it."""
    import gc
    import weakref
    from paper_1611_00463_gb300 import pgs
    ws = _FakeDeviceTensor(0x7000000, 4096)
    st = _FakeDeviceTensor(0x8000000, pgs.STATS_BYTES)
    refs = [weakref.ref(ws), weakref.ref(st)]
    cfg = pgs.make_config(dtype="u64", workspace=ws, stats=st)
    del ws, st
    gc.collect()
    assert all(r() is not None for r in refs)
    assert cfg.workspace == 0x7000000 and cfg.workspace_bytes == 4096 and cfg.stats == 0x8000000
    del cfg
    gc.collect()
    assert all(r() is None for r in refs)


def test_copy_back_option_is_validated():
    from paper_1611_00463_gb300 import pgs
    good = pgs.make_config(dtype="u64", copy_back="end")
    assert pgs.pgs_host_workspace_bytes(1 << 20, 16, good) > 0
    bad = pgs.make_config(dtype="u64")
    bad.copy_back = 3
    assert pgs.pgs_host_workspace_bytes(1 << 20, 16, bad) == 0


def test_binding_structs_match_the_c_compiler():
    """Every field of the binding's ctypes structs sits at the offset, and every
    struct has the size, that the C compiler gives them from include/pgs.h."""
    import os
    import shutil
    import subprocess
    import tempfile
    from paper_1611_00463_gb300 import pgs
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = {"pgs_config": pgs.pgs_config, "pgs_stats": pgs.pgs_stats, "pgs_launch_record": pgs.pgs_launch_record}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pgs.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([cc, "-I", os.path.join(root, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_static_limits_match_header_and_every_option_fits(lib):
    """pgs_sort_static promises that every option combination fits its scratch
    array within its n and P limits: the workspace the same sort would need
    (host-only size query, payload included) stays within the array for every
    key type, splitter mode, merge width, exchange, sample count and size."""
    import itertools
    from paper_1611_00463_gb300 import pgs
    hdr = open(os.path.join(ROOT, "include", "pgs.h")).read()
    assert re.search(r"#define PGS_STATIC_MAX_KEYS \(1u << 16\)", hdr) and pgs.STATIC_MAX_KEYS == 1 << 16
    assert re.search(r"#define PGS_STATIC_MAX_P 64u", hdr) and pgs.STATIC_MAX_P == 64
    assert re.search(r"#define PGS_STATIC_SCRATCH_BYTES \(8u << 20\)", hdr) and pgs.STATIC_SCRATCH_BYTES == 8 << 20
    worst = 0
    for dt, spl, mw, ex, g, s, eps in itertools.product(["u32", "u64", "f32"], ["sampled", "learned"], [2, 4],
                                                        ["auto", "scatter"], [False, True], [0, 1, 4097, 2**32 - 1],
                                                        [0.0, 1e-6]):
        cfg = pgs.make_config(dtype=dt, splitters=spl, merge_ways=mw, exchange=ex, guaranteed=g,
                              samples_per_run=s, eps=eps)
        for n in [1 << 16, (1 << 16) - 1, 60_000, 4353, 4352 * 8 + 1, 1]:
            for P in [64, 63, 33, 2, 1]:
                b = pgs.pgs_workspace_bytes(n, P, cfg)
                assert 0 < b <= pgs.STATIC_SCRATCH_BYTES, (dt, spl, mw, ex, g, s, eps, n, P, b)
                worst = max(worst, b)
    assert worst > pgs.STATIC_SCRATCH_BYTES // 2        # the grid reaches the expensive combinations


@pytest.mark.parametrize("P", [2, 16, 63])
@pytest.mark.parametrize("dtype", ["u32", "u64"])
def test_bucket_rounds_planned_ahead_only_within_their_limit(P, dtype):
    """A single sort with pairwise rounds whose every bucket round is small
    (ceil(n / 1088) + P^2 <= 4096 tiles) has its bucket rounds planned by the
    offsets kernel, in job tables of its own: its workspace holds them up to
    that n and not one key past it, and never with four-way rounds."""
    from paper_1611_00463_gb300 import pgs
    limit = (4096 - P * P) * 1088
    cfg = pgs.make_config(dtype=dtype, merge_ways=2)
    rounds = (P - 1).bit_length()
    tables = rounds * ((limit + 1087) // 1088 + P * P) * 48     # at least the job tables
    assert pgs.pgs_workspace_bytes(limit, P, cfg) - pgs.pgs_workspace_bytes(limit + 1, P, cfg) >= tables
    four = pgs.make_config(dtype=dtype, merge_ways=4)
    assert pgs.pgs_workspace_bytes(limit, P, four) - pgs.pgs_workspace_bytes(limit + 1, P, four) <= 0
