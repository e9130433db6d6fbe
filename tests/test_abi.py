"""The C-ABI library loads and exports every entry point include/wl.h declares
(no GPU needed: nothing here launches work)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2304_08159_gb300 import build, wl

    build.build()
    return wl.load()


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(wl_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2304_08159_gb300 import wl

    assert sorted(wl.EXPORTS) == _declared()


def test_workspace_bytes_host_only(lib):
    from paper_2304_08159_gb300 import wl

    small = wl.wl_workspace_bytes((128, 64))
    o = wl.wl_default_opts()
    o.precision = 0
    big = wl.wl_workspace_bytes((512, 256, 256), o)
    assert small > 0 and big > 0
    # 3 velocity buffers + (3 coefficients + z, x, x2) on the fine level, + about 1/7 for coarse levels
    nc = 512 * 256 * 256
    assert 4 * nc * (9 + 6) <= big <= 4 * nc * (9 + 6 * 8 / 7) + (1 << 20)
    # NULL options mean the defaults: the double-float pressure adds ph, pl and the residual
    assert wl.wl_workspace_bytes((512, 256, 256)) == wl.wl_workspace_bytes((512, 256, 256), wl.wl_default_opts())
    assert wl.wl_workspace_bytes((512, 256, 256)) - big == 3 * 4 * nc
    # 16-bit coarse levels add 16-bit copies of their D coefficient fields and hold z, x, x2
    # in 2 bytes instead of 4 (in 3-D the two cancel exactly); level 1 adds an FP32 staging
    # field for the restricted fine residual
    o.coarse_precision = wl.WL_COARSE_BF16
    assert wl.wl_workspace_bytes((512, 256, 256), o) == big + 4 * nc // 8
    o.coarse_precision = 3
    assert wl.wl_workspace_bytes((512, 256, 256), o) == 0
    assert wl.wl_workspace_bytes((1, 64)) == 0
    assert wl.wl_workspace_bytes((8,)) == 0


def test_default_opts(lib):
    from paper_2304_08159_gb300 import wl

    o = wl.wl_default_opts()
    assert o.tol == 1e-6 and o.max_vcycles == 32 and o.post == 4 and o.eps == 1.0
    assert o.dt_cap == 10.0 and o.advect == 1 and o.use_graph == 1


def test_product_path_does_not_import_oracle():
    """The library package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2304_08159_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text and "wl_oracle" not in text, f


def test_debug_library_exports_the_same_symbols(lib):
    """The bounds-checked build (libwl_debug.so) exports every declared entry point too."""
    import ctypes

    from paper_2304_08159_gb300 import build, wl

    build.build(debug=True)
    dbg = ctypes.CDLL(wl.DEBUG_LIB_PATH)
    for name in _declared():
        assert hasattr(dbg, name), name


def test_header_constants_match_binding():
    """The binding's kernel classes and path bits are the header's, in the header's order."""
    from paper_2304_08159_gb300 import wl

    text = open(os.path.join(ROOT, "include", "wl.h")).read()
    classes = dict((n, int(v)) for n, v in re.findall(r"#define WL_KCLASS_([A-Z_]+)\s+(\d+)", text))
    count = classes.pop("COUNT")
    assert count == len(wl.KCLASSES) == len(classes)
    assert sorted(classes.values()) == list(range(count))
    for name, idx in classes.items():
        assert wl.KCLASSES[idx] == name.lower(), (name, idx)
    paths = dict((n, int(v)) for n, v in re.findall(r"#define (WL_PATH_[A-Z_]+)\s+(\d+)", text))
    for name, bit in paths.items():
        assert getattr(wl, name) == bit, name
