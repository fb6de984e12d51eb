"""A failed host allocation inside the library is a status, not a crash (CPU only).

The CSR analysis copies the row pointers on the host.  Run in a child process whose address
space is capped just above what it already uses, pk_csr_plan and pk_csr_create cannot make
that copy: both must return PK_ERR_OOM with a message, and the process must go on (no
exception may cross the C boundary, which would abort it)."""
import subprocess
import sys
import textwrap

import pytest

CHILD = textwrap.dedent(r"""
    import ctypes as C, resource, sys
    import numpy as np
    lib = C.CDLL(sys.argv[1])
    lib.pk_last_error.restype = C.c_char_p
    n = 1 << 26                                   # 256 MiB of row pointers, every row empty
    rp = np.zeros(n + 1, dtype=np.int32)
    vm = int(open("/proc/self/statm").read().split()[0]) * resource.getpagesize()
    resource.setrlimit(resource.RLIMIT_AS, (vm + (64 << 20), resource.getrlimit(resource.RLIMIT_AS)[1]))
    stats = (C.c_byte * 4096)()
    st1 = lib.pk_csr_plan(C.c_int64(n), C.c_int64(0), rp.ctypes.data_as(C.c_void_p), C.c_int32(152), stats)
    msg1 = lib.pk_last_error().decode()
    h = C.c_void_p()
    st2 = lib.pk_csr_create(C.c_int64(n), C.c_int64(0), rp.ctypes.data_as(C.c_void_p), None, None,
                            C.c_int32(0), None, C.byref(h))
    msg2 = lib.pk_last_error().decode()
    print(st1, st2, h.value is None, "|", msg1, "|", msg2)
""")


def test_host_allocation_failure_returns_oom():
    if not sys.platform.startswith("linux"):  # pragma: no cover
        pytest.skip("needs /proc and RLIMIT_AS")
    from paper_1410_4054_gb300 import pk

    path = str(pk.lib_path())
    pk.lib()  # builds the library if needed
    r = subprocess.run([sys.executable, "-c", CHILD, path], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    st1, st2, null_handle, rest = r.stdout.split(maxsplit=3)
    assert int(st1) == pk.PK_ERR_OOM and int(st2) == pk.PK_ERR_OOM and null_handle == "True"
    assert rest.count("host memory allocation failed") == 2
