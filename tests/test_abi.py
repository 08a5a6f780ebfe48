"""The C-ABI library loads and exports every entry point that include/dpc.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dpc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dpc_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1606_08150_gb300 import build

    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for fn in ("dpc_sssp", "dpc_spmv_csr", "dpc_tree_descendants", "dpc_tree_height", "dpc_device_init",
               "dpc_status_string", "dpc_sssp_workspace_size", "dpc_spmv_csr_workspace_size",
               "dpc_tree_workspace_size"):
        assert fn in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1606_08150_gb300 import dpc

    assert sorted(dpc.EXPORTS) == declared_functions()


def header_enum(name):
    """Enumerator -> value of `typedef enum name {...}` in the header."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef enum " + name + r"\s*\{(.*?)\}", text, flags=re.S).group(1)
    return {k: int(v) for k, v in re.findall(r"(\w+)\s*=\s*(\d+)", body)}


def test_binding_constants_match_the_header():
    """The binding's level, status and flag constants and the struct sizes are
    the header's."""
    from paper_1606_08150_gb300 import dpc

    levels = header_enum("dpc_level")
    assert {k.lower().replace("dpc_", ""): v for k, v in levels.items()} == dpc.LEVELS
    status = header_enum("dpc_status")
    for k, v in status.items():
        assert getattr(dpc, k.replace("DPC_", "")) == v, k
    text = open(HEADER).read()
    flags = dict(re.findall(r"#define DPC_(FLAG_\w+)\s+(0x[0-9a-fA-F]+)u", text))
    assert flags and all(getattr(dpc, k) == int(v, 16) for k, v in flags.items())
    # the size of the allocation-free entry point's array, (size_t)A << B in the header
    a, b = re.search(r"#define DPC_NOALLOC_SCRATCH_BYTES\s+\(\(size_t\)(\d+)\s*<<\s*(\d+)\)", text).groups()
    assert dpc.NOALLOC_SCRATCH_BYTES == int(a) << int(b)
    assert dpc.MAILBOX_CAP == int(re.search(r"#define DPC_MAILBOX_CAP\s+(\d+)", text).group(1))
    # struct layouts: the C compiler's sizes and offsets against the ctypes mirrors
    import shutil
    import subprocess
    import tempfile

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    fields = [("dpc_tuning", dpc.Tuning), ("dpc_stats", dpc.Stats), ("dpc_job", dpc.Job),
              ("dpc_mailbox", dpc.MailboxLayout)]
    lines = ['#include "dpc.h"', "#include <stdio.h>", "#include <stddef.h>", "int main(void) {"]
    for cname, cls in fields:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), src, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    want = []
    for _, cls in fields:
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f).offset for f, _ in cls._fields_]
    assert got == want


def test_host_only_calls(lib):
    lib.dpc_status_string.restype = ctypes.c_char_p
    assert lib.dpc_status_string(0) == b"DPC_OK"
    assert b"WORKSPACE" in lib.dpc_status_string(2)
    assert lib.dpc_abi_version() == 2
    out = ctypes.c_size_t(0)
    # workspace queries are pure host arithmetic
    for level in range(5):
        assert lib.dpc_spmv_csr_workspace_size(1000, 20000, level, None, ctypes.byref(out)) == 0
        assert out.value >= 256
        assert lib.dpc_sssp_workspace_size(1000, 20000, level, None, ctypes.byref(out)) == 0
        assert lib.dpc_tree_workspace_size(1000, level, None, ctypes.byref(out)) == 0
    assert lib.dpc_spmv_csr_workspace_size(-1, 0, 0, None, ctypes.byref(out)) == 1
    assert lib.dpc_spmv_csr_workspace_size(10, 10, 7, None, ctypes.byref(out)) == 1
    assert lib.dpc_spmv_csr_workspace_size(10, 10, 5, None, ctypes.byref(out)) == 0 and out.value > 256  # queue level
    assert lib.dpc_sssp_workspace_size(1000, 20000, 5, None, ctypes.byref(out)) == 0 and out.value > 256
    assert lib.dpc_tree_workspace_size(1000, 5, None, ctypes.byref(out)) == 0 and out.value > 256
    assert lib.dpc_sssp_workspace_size(0, 0, 0, None, ctypes.byref(out)) == 1
    # the wait diagnostic checks its arguments before launching anything
    word = ctypes.c_uint32(0)
    assert lib.dpc_wait_selftest(ctypes.c_uint32(100), None, None) == 1
    assert lib.dpc_wait_selftest(ctypes.c_uint32(0), ctypes.byref(word), None) == 1
    assert lib.dpc_wait_selftest(ctypes.c_uint32(10_000_001), ctypes.byref(word), None) == 1
    # the gather-rate diagnostic checks its sizes first (a power of two from 32 to 2^26)
    g = ctypes.c_int64(0)
    fake = ctypes.c_void_p(0x1000)
    lib.dpc_gather_rate.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]
    assert lib.dpc_gather_rate(fake, 1000, 1, fake, ctypes.byref(g), None) == 1
    assert lib.dpc_gather_rate(fake, 1 << 27, 1, fake, ctypes.byref(g), None) == 1
    assert lib.dpc_gather_rate(fake, 1 << 20, 0, fake, ctypes.byref(g), None) == 1
    assert lib.dpc_gather_rate(None, 1 << 20, 1, fake, ctypes.byref(g), None) == 1
    for level in range(6):
        assert lib.dpc_pagerank_workspace_size(1000, 20000, level, None, ctypes.byref(out)) == 0
        assert out.value > 256 + 2 * 4000
    assert lib.dpc_pagerank_workspace_size(0, 0, 0, None, ctypes.byref(out)) == 1
    # the accessibility query: a null pointer is simply not accessible; a null result is refused
    flag = ctypes.c_int32(7)
    lib.dpc_memory_device_accessible.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.dpc_memory_device_accessible(None, ctypes.byref(flag)) == 0 and flag.value == 0
    assert lib.dpc_memory_device_accessible(fake, None) == 1


def test_argument_errors_return_before_any_cuda_call(lib):
    P = ctypes.c_void_p
    fake = P(0x1000)
    # negative sizes, a bad level, null outputs, missing workspace: all rejected on the host
    assert lib.dpc_spmv_csr(fake, fake, fake, -1, 4, 4, fake, fake, 4, None, fake, 1 << 20, None, None) == 1
    assert lib.dpc_spmv_csr(fake, fake, fake, 4, 4, 4, fake, None, 4, None, fake, 1 << 20, None, None) == 1
    assert lib.dpc_spmv_csr(fake, fake, fake, 4, 4, 4, fake, fake, 9, None, fake, 1 << 20, None, None) == 1
    assert lib.dpc_spmv_csr(fake, fake, fake, 4, 4, 4, fake, fake, 4, None, None, 0, None, None) == 2
    assert lib.dpc_spmv_csr(fake, fake, fake, 4, 4, 4, fake, fake, 4, None, fake, 16, None, None) == 2
    assert lib.dpc_sssp(fake, fake, fake, 4, 4, 4, fake, 4, None, fake, 1 << 20, None, None) == 1  # source == n
    assert lib.dpc_sssp(fake, fake, fake, 4, 4, -1, fake, 4, None, fake, 1 << 20, None, None) == 1
    assert lib.dpc_tree_height(fake, fake, 4, 5, fake, 4, None, fake, 1 << 20, None, None) == 1  # root >= n
    assert lib.dpc_tree_descendants(fake, None, 4, 0, fake, 4, None, fake, 1 << 20, None, None) == 1
    pr = lib.dpc_pagerank
    pr.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_int32, P, ctypes.c_int,
                   P, P, ctypes.c_size_t, P, P]
    assert pr(fake, fake, fake, 4, 4, 1.5, 3, fake, 4, None, fake, 1 << 20, None, None) == 1  # damping > 1
    assert pr(fake, fake, fake, 4, 4, float("nan"), 3, fake, 4, None, fake, 1 << 20, None, None) == 1
    assert pr(fake, fake, fake, 4, 4, 0.85, -1, fake, 4, None, fake, 1 << 20, None, None) == 1
    assert pr(fake, None, fake, 4, 4, 0.85, 3, fake, 4, None, fake, 1 << 20, None, None) == 1  # m > 0, no sources
    assert pr(fake, fake, fake, 4, 4, 0.85, 3, fake, 4, None, fake, 16, None, None) == 2  # workspace too small


def test_binding_refuses_host_memory_the_device_cannot_read():
    """SpMV's matrix arrays may be pinned host memory the device reads in
    place; pageable host memory, and x or y on the host, are refused before
    any call into the library."""
    import torch

    from paper_1606_08150_gb300 import dpc

    off = torch.tensor([0, 1, 2], dtype=torch.int32)
    col = torch.tensor([0, 1], dtype=torch.int32)
    val = torch.ones(2, dtype=torch.float32)
    x = torch.ones(2, dtype=torch.float32)
    y = torch.empty(2, dtype=torch.float32)
    with pytest.raises(ValueError):
        dpc.spmv_csr(off, col, val, x, y, "grid", workspace=torch.empty(1 << 16, dtype=torch.uint8))


def test_bad_tuning_rejected(lib):
    from paper_1606_08150_gb300 import dpc

    out = ctypes.c_size_t(0)
    t = dpc.Tuning(parent_threads=100)
    assert lib.dpc_spmv_csr_workspace_size(100, 100, 4, ctypes.byref(t), ctypes.byref(out)) == 1
    t = dpc.Tuning(chunk=-5)
    assert lib.dpc_spmv_csr_workspace_size(100, 100, 4, ctypes.byref(t), ctypes.byref(out)) == 1


def test_mailbox_host_side(lib):
    """The mailbox calls are host code: posting fills the ring in order and
    publishes the count, a full ring (DPC_MAILBOX_CAP posted, none taken) is
    refused, stop sets the flag; bad arguments are rejected."""
    from paper_1606_08150_gb300 import dpc

    mb = dpc.MailboxLayout()
    P = ctypes.c_void_p
    lib.dpc_mailbox_init.argtypes = [P]
    lib.dpc_mailbox_post.argtypes = [P, P, ctypes.c_int32]
    lib.dpc_mailbox_stop.argtypes = [P]
    lib.dpc_mailbox_taken.argtypes = [P, P]
    addr = ctypes.addressof(mb)
    mb.posted = 99
    assert lib.dpc_mailbox_init(addr) == 0 and mb.posted == 0 and mb.taken == 0 and mb.stop == 0
    for i in range(dpc.MAILBOX_CAP):
        job = dpc.Job(dpc.JOB_SSSP, 10 + i, 20, i % 7, 0x1000, 0x2000, 0x3000, 0x4000)
        assert lib.dpc_mailbox_post(addr, ctypes.byref(job), i % 5) == 0
    assert mb.posted == dpc.MAILBOX_CAP
    assert [mb.jobs[i].n for i in (0, 1, dpc.MAILBOX_CAP - 1)] == [10, 11, 10 + dpc.MAILBOX_CAP - 1]
    assert mb.slots[7] == 2 and mb.jobs[7].source == 0
    job = dpc.Job(dpc.JOB_SSSP, 1, 0, 0, 0x1000, 0, 0, 0x4000)
    assert lib.dpc_mailbox_post(addr, ctypes.byref(job), 0) == dpc.ERR_OVERFLOW  # ring full
    mb.taken = 3  # the kernel admitted three: room for three more, in the ring's first entries
    assert lib.dpc_mailbox_post(addr, ctypes.byref(job), 4) == 0
    assert mb.posted == dpc.MAILBOX_CAP + 1 and mb.jobs[0].n == 1 and mb.slots[0] == 4
    got = ctypes.c_uint64(0)
    assert lib.dpc_mailbox_taken(addr, ctypes.byref(got)) == 0 and got.value == 3
    assert lib.dpc_mailbox_stop(addr) == 0 and mb.stop == 1
    assert lib.dpc_mailbox_post(addr, None, 0) == dpc.ERR_INVALID_ARG
    assert lib.dpc_mailbox_post(addr, ctypes.byref(job), -1) == dpc.ERR_INVALID_ARG
    assert lib.dpc_mailbox_init(None) == dpc.ERR_INVALID_ARG


def test_engine_serve_rejects_bad_arguments_on_the_host(lib):
    """dpc_engine_serve checks its scalars and pointers before any CUDA call."""
    from paper_1606_08150_gb300 import dpc

    P = ctypes.c_void_p
    lib.dpc_engine_serve.argtypes = [P, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P,
                                     ctypes.c_uint32, P, P, P]
    mb = dpc.MailboxLayout()
    state = (ctypes.c_int32 * 4)()
    ws = P(0x1000)
    args = dict(ws=ws, bytes=1 << 30, slots=4, max_n=100, max_m=100, tun=None, mb=ctypes.addressof(mb), limit=1000,
                state=ctypes.addressof(state))

    def call(**kw):
        a = dict(args, **kw)
        return lib.dpc_engine_serve(a["ws"], a["bytes"], a["slots"], a["max_n"], a["max_m"], a["tun"], a["mb"],
                                    a["limit"], a["state"], None, None)

    assert call(slots=0) == dpc.ERR_INVALID_ARG
    assert call(max_n=0) == dpc.ERR_INVALID_ARG
    assert call(mb=None) == dpc.ERR_INVALID_ARG
    assert call(state=None) == dpc.ERR_INVALID_ARG
    assert call(limit=0) == dpc.ERR_INVALID_ARG
    assert call(limit=10_000_001) == dpc.ERR_INVALID_ARG
    assert call(ws=None) == dpc.ERR_WORKSPACE
