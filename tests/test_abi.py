"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point declared in include/spkmc.h, and its host-only entry points
(rate table, validation, sizes) behave as declared.  No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1005_4713_gb300 as sp
from paper_1005_4713_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "spkmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(spkmc_[a-z_0-9]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(_abi.PROTOTYPES)


def test_library_exports_every_declared_symbol():
    lib = sp.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm103a():
    from paper_1005_4713_gb300 import build
    out = os.popen(f"strings -a {build.LIB} | grep -c sm_103a").read().strip()
    assert int(out or 0) > 0


def test_rate_table_bitwise_equal_to_oracle():
    for J, H, T in [(1.0, 0.0, 4.5115), (1.0, 0.01, 4.43), (-0.5, 0.2, 2.0), (1.0, 0.0, 0.01)]:
        assert np.array_equal(sp.spkmc_rate_table(J, H, T), oracle.rates(J, H, T))


def test_rmax_bounds_bitwise_equal_to_oracle():
    """The library takes the bounds from its rate table; the oracle evaluates
    the prescribed formula of Sec. 3.2 directly.  Same bits."""
    for d in (2, 4, 8, 16):
        for J, H, T in [(1.0, 0.0, 4.5115), (1.0, 0.01, 4.43), (-0.5, 0.2, 2.0), (1.0, -0.3, 0.01),
                        (0.0, 0.0, 3.0), (2.0, 0.0, 1e6)]:
            assert sp.spkmc_rmax_bounds(d, J, H, T) == oracle.rmax_bounds(d, J, H, T)


@pytest.mark.parametrize("d,T", [(3, 1.0), (32, 1.0), (4, 0.0), (4, float("nan"))])
def test_rmax_bounds_rejects_bad_arguments(d, T):
    with pytest.raises(sp.SpkmcError) as e:
        sp.spkmc_rmax_bounds(d, 1.0, 0.0, T)
    assert e.value.code == sp.SPKMC_EINVAL


def test_two_colour_sizes_and_invalid_combinations():
    # two colours: K/2 active domains, so four times the scratch of eight
    p8 = sp.make_params(64, 8)
    p2 = sp.make_params(64, 8, sublattice=sp.SPKMC_SUBLATTICE_2_RANDOM)
    K = 8 ** 3
    assert sp.spkmc_bytes_required(p2) - sp.spkmc_bytes_required(p8) == (K // 2 - K // 8) * 192
    for bad in (sp.make_params(16, 4, sublattice=2), sp.make_params(16, 4, sublattice=-1),
                sp.make_params(16, 4, sublattice=1, rmax_mode=sp.SPKMC_RMAX_LEARNED)):
        assert sp.spkmc_bytes_required(bad) == 0
        with pytest.raises(sp.SpkmcError) as e:
            sp.spkmc_create_ex(bad)
        assert e.value.code == sp.SPKMC_EINVAL


@pytest.mark.parametrize("mode", [-1, 3])
def test_create_rejects_unknown_rmax_mode(mode):
    p = sp.make_params(16, 4, rmax_mode=mode)
    assert sp.spkmc_bytes_required(p) == 0
    with pytest.raises(sp.SpkmcError) as e:
        sp.spkmc_create_ex(p)
    assert e.value.code == sp.SPKMC_EINVAL
    assert "rmax_mode" in sp.spkmc_last_error()


@pytest.mark.parametrize("J,H,T", [(1.0, 0.0, 0.0), (1.0, 0.0, -1.0), (float("nan"), 0.0, 1.0),
                                   (1.0, float("inf"), 1.0), (1.0, 0.0, float("inf"))])
def test_rate_table_rejects_bad_arguments(J, H, T):
    with pytest.raises(sp.SpkmcError) as e:
        sp.spkmc_rate_table(J, H, T)
    assert e.value.code == sp.SPKMC_EINVAL


@pytest.mark.parametrize("L,d", [(16, 3), (16, 32), (12, 4), (10, 2), (16, 16), (0, 4), (-8, 2)])
def test_create_rejects_invalid_geometry_before_touching_the_gpu(L, d):
    with pytest.raises(sp.SpkmcError) as e:
        sp.spkmc_create(L, d, 1.0, 0.0, 4.5, 1)
    assert e.value.code == sp.SPKMC_EINVAL
    assert "domain edge" in sp.spkmc_last_error() or "L" in sp.spkmc_last_error()


def test_create_rejects_bad_temperature():
    with pytest.raises(sp.SpkmcError) as e:
        sp.spkmc_create(16, 4, 1.0, 0.0, 0.0, 1)
    assert e.value.code == sp.SPKMC_EINVAL


@pytest.mark.parametrize("L,d", [(16, 8), (24, 4), (48, 8), (96, 16), (128, 16), (1024, 16), (20, 2), (4, 2)])
def test_resolve_domain_edge(L, d):
    assert sp.spkmc_resolve_domain_edge(L) == d


def test_resolve_domain_edge_none():
    assert sp.spkmc_resolve_domain_edge(6) == 0


def test_bytes_required():
    p = sp.make_params(1024, 16)
    # domain blocks: rows (L^3/8 bytes) and 6 ghost faces of d 16-bit words;
    # counts: 64 B per domain; scratch: 192 B per active domain; the table
    # of products fl(n r_c), 14 x (d^3 + 1) doubles rounded up to 256 B
    K = 64 ** 3
    table = -(-14 * (16 ** 3 + 1) * 8 // 256) * 256
    expect = 1024 ** 3 // 8 + K * 6 * 16 * 2 + K * 64 + (K // 8) * 192 + table
    assert sp.spkmc_bytes_required(p) == expect
    assert sp.spkmc_bytes_required(sp.make_params(16, 3)) == 0


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """ctypes mirrors of the header structs have the C compiler's sizes and offsets."""
    import subprocess
    structs = {
        "spkmc_params": _abi.spkmc_params, "spkmc_config": _abi.spkmc_config,
        "spkmc_obs": _abi.spkmc_obs, "spkmc_event": _abi.spkmc_event,
        "spkmc_state": _abi.spkmc_state, "spkmc_info": _abi.spkmc_info,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "spkmc.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)


def build_abi_example(tmp_path):
    """tests/abi_example.c compiled and linked against the in-tree library."""
    import subprocess
    exe = tmp_path / "abi_example"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "abi_example.c"), "-L", os.path.dirname(_abi.LIB_PATH), "-lspkmc",
                    "-Wl,-rpath," + os.path.dirname(_abi.LIB_PATH), "-o", str(exe)], check=True)
    return str(exe)


def test_c_program_links_and_fails_loudly_without_a_device(tmp_path):
    import subprocess
    import torch
    exe = build_abi_example(tmp_path)
    bad = subprocess.run([exe, "1"], capture_output=True, text=True)
    assert bad.returncode == 2 and "usage" in bad.stderr
    bad = subprocess.run([exe, "30", "8", "1", "0", "4.5", "1", "10"], capture_output=True, text=True)
    assert bad.returncode == 1 and bad.stdout == ""
    assert "spkmc_create" in bad.stderr  # L % (2d) != 0, or no device: the create call fails first
    if not torch.cuda.is_available():
        r = subprocess.run([exe], capture_output=True, text=True)
        assert r.returncode == 1 and r.stdout == ""
        assert "no CUDA device" in r.stderr
