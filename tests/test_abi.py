"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/burr.h declares (host-only calls; no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "burr.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(burr_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_12365_gb300 import build as B
    path = B.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    fns = declared_functions()
    for f in ("burr_build", "burr_query", "burr_free", "burr_export", "burr_default_params"):
        assert f in fns


def test_every_declared_symbol_is_exported(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2411_12365_gb300 import burr
    assert sorted(burr.EXPORTED) == declared_functions()


def test_default_params_layout(lib):
    from paper_2411_12365_gb300 import burr
    burr.load(os.path.join(ROOT, "paper_2411_12365_gb300", "_lib", "libburr.so"))
    p = burr.default_params()
    assert C.sizeof(burr.Params) == 96
    assert (p.ribbon_width, p.bucket_slots, p.layers, list(p.levels)) == (64, 128, 4, [0, 32, 64, 128])
    assert p.load_factor == 1.015 and p.partition_slots == 65536 and p.fallback_max_retries == 16
    assert p.lower_partition_slots == 4096 and p.min_partition_slots == 4096
    assert p.cut_search == burr.CUT_NONE and p.cut_search_range == 50
    # the oracle's defaults are the same workload
    from oracle import oracle as O
    q = O.default_params()
    assert (q.alpha, q.partition_slots, q.min_partition_slots, q.seed, q.layers, q.fb_slack,
            q.lower_partition_slots, q.cut_search, q.cut_search_range) == \
        (p.load_factor, p.partition_slots, p.min_partition_slots, p.seed, p.layers, p.fallback_slack,
         p.lower_partition_slots, p.cut_search, p.cut_search_range)


def test_strerror(lib):
    lib.burr_strerror.restype = C.c_char_p
    assert lib.burr_strerror(-3).decode().startswith("unsolvable")


def test_server_rejects_bad_config_without_touching_the_device(lib):
    from paper_2411_12365_gb300 import burr
    burr.load(os.path.join(ROOT, "paper_2411_12365_gb300", "_lib", "libburr.so"))
    for budget, kw in ((0, {}), (1 << 30, dict(partition_slots=0))):
        with pytest.raises(burr.BurrError) as e:
            burr.Server(budget, **kw)
        assert e.value.code == burr.ERR_INVALID


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes structures have the sizes the C compiler gives the header's."""
    from paper_2411_12365_gb300 import burr
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "burr.h"\nint main(void) { printf("%zu %zu %zu %zu %zu\\n", '
                   "sizeof(burr_params), sizeof(burr_stats_t), sizeof(burr_server_config), "
                   "sizeof(burr_server_stats_t), sizeof(burr_layer_geometry_t)); return 0; }\n")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == [C.sizeof(burr.Params), C.sizeof(burr.Stats), C.sizeof(burr.ServerConfig),
                   C.sizeof(burr.ServerStats), C.sizeof(burr.LayerGeometry)]


def test_allocator_hook_arguments_without_the_device(lib):
    from paper_2411_12365_gb300 import burr
    burr.load(os.path.join(ROOT, "paper_2411_12365_gb300", "_lib", "libburr.so"))
    with pytest.raises(ValueError):
        burr.set_allocator(alloc=lambda n, s: 0)
    L = burr.load()
    with pytest.raises(burr.BurrError):                       # one of the pair missing
        burr._check(L.burr_set_allocator(burr._ALLOC_FN(lambda n, s, c: None), burr._FREE_FN(), None))
    calls = []
    burr.set_allocator(lambda n, s: calls.append(n) or 0, lambda p, s: None)   # nothing held: accepted
    burr.set_allocator(None, None)
    assert calls == []                                        # installing allocates nothing
