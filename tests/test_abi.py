"""The C-ABI library loads and exports every entry point include/pgc.h declares; configuration
checks run on the host (no GPU needed).  Also checks that the oracle and the CUDA library share
no code."""
import ctypes as C
import os
import re

import pytest

from paper_2404_19602_gb300 import build, pgc
from paper_2404_19602_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return pgc.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "pgc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pgc_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "pgc_init" in names and "pgc_step" in names and "pgc_moments" in names
    assert "pgc_reconstruct_f" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in pgc.SIGNATURES, n


def test_query_sizes_default(lib):
    cfg = pgc.pgc_config_default()
    s = pgc.pgc_query_sizes(cfg)
    assert s["P"] == 1 and s["Q"] == 1
    assert s["state_bytes"] == 2 * 1 * 10048 * 4
    assert s["hist_bytes"] >= 3 * 240 * 240 * 4


def test_query_sizes_gpc_shapes(lib):
    from paper_2404_19602_gb300 import workloads as W

    s = pgc.pgc_query_sizes(pgc.config_from(W.GAP_UQ_1E6))
    assert (s["P"], s["Q"]) == (6, 6)
    assert s["state_bytes"] == 2 * 6 * 1_000_000 * 4
    s = pgc.pgc_query_sizes(pgc.config_from(W.GAP_FIELD_UQ_4E6))
    assert (s["P"], s["Q"]) == (21, 36)
    s = pgc.pgc_query_sizes(pgc.config_from(W.scaled(W.GAP_UQ_1E6, precision="fp64")))
    assert s["state_bytes"] == 2 * 6 * 1_000_000 * 8


@pytest.mark.parametrize("field,value", [("n_particles", 0), ("dt_fs", 0.0), ("Nk", 1), ("precision", 7),
                                         ("pauli_norm", 5), ("n_theta_edge", 63), ("mech_mask", 64),
                                         ("max_outputs", 0)])
def test_invalid_configs_are_rejected(lib, field, value):
    cfg = pgc.pgc_config_default()
    setattr(cfg, field, value)
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_query_sizes(cfg)
    assert e.value.status == pgc.PGC_EINVAL
    assert lib.pgc_last_error(None)


@pytest.mark.parametrize("M,quad", [(7, 8), (3, 5), (31, 32)])
def test_uncompiled_shape_is_unsupported(lib, M, quad):
    cfg = pgc.pgc_config_default()
    cfg.eps0_eV.lo, cfg.eps0_eV.hi = 0.05, 0.15
    cfg.degree_M, cfg.quad_per_dim = M, quad
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_query_sizes(cfg)
    assert e.value.status in (pgc.PGC_EUNSUPPORTED, pgc.PGC_EINVAL)


@pytest.mark.parametrize("M", [0, 1, 2, 3, 4, 5, 6, 8, 10, 12, 15, 20, 25, 30])
def test_one_dimensional_degrees_are_compiled(lib, M):
    cfg = pgc.pgc_config_default()
    cfg.eps0_eV.lo, cfg.eps0_eV.hi = 0.05, 0.15
    cfg.degree_M, cfg.quad_per_dim = M, M + 1
    s = pgc.pgc_query_sizes(cfg)
    assert s["P"] == s["Q"] == M + 1


def test_init_rejects_null_buffers(lib):
    cfg = pgc.pgc_config_default()
    out = C.c_void_p()
    st = lib.pgc_init(C.byref(cfg), None, None, None, None, None, C.byref(out))
    assert st == pgc.PGC_EINVAL and not out.value


def test_oracle_and_library_share_no_code():
    pkg = os.path.join(ROOT, "paper_2404_19602_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "pgc_oracle" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2404_19602_gb300" not in txt, f
            assert "pgc.h" not in txt and "csrc" not in txt, f


def test_band_minimum_law_fields_are_checked(lib):
    """The width law needs a positive, ordered width interval; an unknown law is rejected."""
    cfg = pgc.pgc_config_default()
    cfg.eps0_law = 7
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_query_sizes(cfg)
    assert e.value.status == pgc.PGC_EINVAL
    cfg = pgc.pgc_config_default()
    cfg.eps0_law = pgc.PGC_EPS0_WIDTH
    cfg.width_nm.lo, cfg.width_nm.hi = 0.0, 0.0
    with pytest.raises(pgc.PgcError):
        pgc.pgc_query_sizes(cfg)
    cfg.width_nm.lo, cfg.width_nm.hi = 7.5, 6.5
    with pytest.raises(pgc.PgcError):
        pgc.pgc_query_sizes(cfg)
    cfg.width_nm.lo, cfg.width_nm.hi = 6.5, 7.5
    s = pgc.pgc_query_sizes(cfg)
    assert (s["P"], s["Q"]) == (6, 6)
    cfg.width_nm.hi = 6.5                      # a deterministic width: no random input
    s = pgc.pgc_query_sizes(cfg)
    assert (s["P"], s["Q"]) == (1, 1)


def test_splitting_field_is_checked(lib):
    cfg = pgc.pgc_config_default()
    assert cfg.splitting == pgc.PGC_SPLIT_LIE
    cfg.splitting = 5
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_query_sizes(cfg)
    assert e.value.status == pgc.PGC_EINVAL
    cfg.splitting = pgc.PGC_SPLIT_STRANG
    assert pgc.pgc_query_sizes(cfg)["P"] == 1


def test_tensor_core_switch_is_checked(lib):
    """tc_proj: an unknown value is invalid; the tensor-core reconstruction exists for the FP32
    21 x 36 shape only."""
    cfg = pgc.pgc_config_default()
    assert cfg.tc_proj == pgc.PGC_TC_OFF
    cfg.tc_proj = 3
    with pytest.raises(pgc.PgcError) as e:
        pgc.pgc_query_sizes(cfg)
    assert e.value.status == pgc.PGC_EINVAL
    cfg.tc_proj = pgc.PGC_TC_F16X3
    with pytest.raises(pgc.PgcError) as e:        # the default shape is 1 x 1
        pgc.pgc_query_sizes(cfg)
    assert e.value.status == pgc.PGC_EUNSUPPORTED
    for mode in (pgc.PGC_TC_F16X3, pgc.PGC_TC_F16):
        c = pgc.config_from(W.scaled(W.GAP_FIELD_UQ_4E6, N=1000, tc_proj=mode))
        s = pgc.pgc_query_sizes(c)
        assert (s["P"], s["Q"]) == (21, 36)
        c.precision = pgc.PGC_FP64
        with pytest.raises(pgc.PgcError) as e:
            pgc.pgc_query_sizes(c)
        assert e.value.status == pgc.PGC_EUNSUPPORTED


def test_plain_c_consumer_compiles_links_and_queries(lib, tmp_path):
    """The header is plain C99 (no C++ constructs), and a C program linked against the library
    can fill a default configuration and query the buffer sizes without a GPU."""
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    src = tmp_path / "consumer.c"
    src.write_text(r'''
#include <stdio.h>
#include "pgc.h"
int main(void)
{
    pgc_config c;
    size_t s = 0, h = 0, w = 0;
    int32_t P = 0, Q = 0;
    pgc_config_default(&c);
    c.eps0_eV.lo = 0.05; c.eps0_eV.hi = 0.15; c.degree_M = 5; c.quad_per_dim = 6; c.n_particles = 1000;
    if (pgc_query_sizes(&c, &s, &h, &w, &P, &Q) != PGC_OK) { puts(pgc_last_error(NULL)); return 1; }
    printf("%d %d %zu\n", P, Q, s);
    c.splitting = 7;
    return pgc_query_sizes(&c, &s, &h, &w, &P, &Q) == PGC_EINVAL ? 0 : 2;
}
''')
    exe = tmp_path / "consumer"
    libdir = os.path.dirname(build.LIB)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I" + os.path.join(ROOT, "include"),
                           str(src), "-o", str(exe), "-L" + libdir, "-lpgc", "-Wl,-rpath," + libdir])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.split() == ["6", "6", str(2 * 6 * 1024 * 4)]
