"""CPU-side checks of the C ABI: the library builds/loads and exports every
entry point that include/dtws.h declares; host-only calls behave."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dtws.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dtws_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_10302_gb300 import build, dtws
    try:
        build.build()
    except (OSError, subprocess.CalledProcessError) as e:  # no nvcc here
        pytest.skip(f"cannot build libdtws.so: {e}")
    return dtws.load()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("dtws_create", "dtws_destroy", "dtws_query", "dtws_query_batch",
                 "dtws_sync_status", "dtws_strerror", "dtws_last_stats", "dtws_set_options"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1812_10302_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (dtws_[a-z0-9_]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)


def test_binding_covers_every_declared_symbol():
    from paper_1812_10302_gb300 import dtws
    assert sorted(dtws.exported_symbols()) == _declared()


def test_default_options_and_strerror(lib):
    from paper_1812_10302_gb300 import dtws
    o = dtws.dtws_default_options()
    assert o.delta == pytest.approx(2.0 ** -10)
    assert o.alpha_per_m == pytest.approx(1e-6)
    assert o.seed_random == 4 and o.seed_proposals == 16 and o.proxy_terms == 16
    assert o.wait_limit_ns == 2_000_000_000
    assert dtws.strerror(dtws.DTWS_EINVAL) == "invalid argument"
    assert dtws.strerror(dtws.DTWS_EOVERFLOW).startswith("more near-ties")


def _c_layout(tmp_path, struct, fields):
    """sizeof and offsetof of each field as a C compiler lays the header's struct out."""
    src = tmp_path / f"{struct}.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "dtws.h"\nint main(void) {\n'
                   f'    printf("%zu\\n", sizeof({struct}));\n' +
                   "".join(f'    printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields) +
                   "    return 0;\n}\n")
    exe = tmp_path / struct
    try:
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                       capture_output=True)
    except (OSError, subprocess.CalledProcessError) as e:
        pytest.skip(f"no C compiler: {e}")
    return [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]


@pytest.mark.parametrize("struct", ["dtws_options", "dtws_query_stats", "dtws_adam"])
def test_binding_structs_match_the_header_layout(struct, tmp_path):
    """The binding's ctypes mirror of each ABI struct has the header's size
    and every field at the header's offset."""
    import ctypes
    from paper_1812_10302_gb300 import dtws
    cls = getattr(dtws, struct)
    fields = [f for f, _ in cls._fields_]
    got = _c_layout(tmp_path, struct, fields)
    assert got[0] == ctypes.sizeof(cls)
    assert got[1:] == [getattr(cls, f).offset for f in fields]


def test_option_defaults(lib):
    from ctypes import sizeof as ctypes_sizeof
    from paper_1812_10302_gb300 import dtws
    o = dtws.dtws_default_options()
    assert (o.ordering, o.timing, o.exact_envelope, o.batch_lanes, o.batch_graph, o.exclusion_zone,
            o.unnormalised, o.rng_seed) == (dtws.DTWS_ORDER_PLAIN, 0, 1, 4, 1, 0, 0, 0)
    # the new field filled the padding before wait_limit_ns: the struct did not grow
    assert ctypes_sizeof(dtws.dtws_options) == 64


def test_create_rejects_bad_arguments_without_device_work(lib):
    import ctypes
    from paper_1812_10302_gb300 import dtws
    h = ctypes.c_void_p()
    assert lib.dtws_create(None, 100, None, ctypes.byref(h)) == dtws.DTWS_EINVAL
    assert lib.dtws_create(ctypes.c_void_p(16), 1, None, ctypes.byref(h)) == dtws.DTWS_EINVAL
    assert lib.dtws_create(ctypes.c_void_p(16), 100, None, None) == dtws.DTWS_EINVAL
    assert lib.dtws_destroy(None) == dtws.DTWS_EINVAL
    assert lib.dtws_query(None, None, 10, 1, 1, None, None, None) == dtws.DTWS_EINVAL


def test_package_has_no_cpu_fallback():
    """The product modules never import the oracle."""
    pkg = os.path.join(ROOT, "paper_1812_10302_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
