"""The C ABI library builds for sm_103a, loads, and exports every symbol declared in include/pyro.h
(no compute call: this runs without a GPU)."""
import os
import re
import ctypes

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "pyro.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(pyro_[a-z_]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol():
    from paper_2603_14040_b300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(lib, s), s
    import paper_2603_14040_b300 as P
    assert sorted(P.EXPORTED) == syms


def test_host_logic_without_gpu():
    import paper_2603_14040_b300 as P
    assert P.lib().pyro_version().startswith(b"pyro-b300")
    assert P.lib().pyro_strerror(-4) == b"non-finite input or iterate"
    o = P.default_opts()
    assert (o.nu1, o.nu2, o.restart_m, o.prec, o.coarsest_min) == (2, 2, 30, P.PREC_MIXED, 4)
    # footprint: degenerate sizes are rejected; odd and coarse-unfriendly sizes are served (their
    # coarsest level is smoothed instead of inverted, so it needs no dense inverse)
    assert P.footprint(1, 8) == 0 and P.footprint(8, 0) == 0
    assert P.footprint(3, 8) > 0 and P.footprint(100, 100) > 0
    assert P.footprint(100, 100) < P.footprint(128, 128)
    f1, f2 = P.footprint(512, 512), P.footprint(1024, 1024)
    assert 3.5 < f2 / f1 < 4.5
    o64 = P.default_opts(prec=P.PREC_FP64)
    assert P.footprint(1024, 1024, o64) > f2
    o10 = P.default_opts(restart_m=10)
    assert P.footprint(1024, 1024, o10) < f2


@pytest.mark.parametrize("kw", [dict(smoother=9), dict(accel=-1), dict(prec=5), dict(eta_coarsen=2), dict(restart_m=0),
                                dict(restart_m=257), dict(nu1=0, nu2=0), dict(nu1=-1), dict(omega_v=0.0),
                                dict(omega_v=2.0), dict(alpha_p=0.0), dict(aa_beta=0.0), dict(aa_beta=1.5),
                                dict(kcycle=17), dict(tile_fusion=5), dict(tile_sweeps=3), dict(tile_fusion64=2),
                                dict(ras_inner=0), dict(max_iter=0), dict(coarsen_ratio=1.2), dict(coarse_sweeps=0),
                                dict(cont_iters=0), dict(coarsest_min=0),
                                dict(gram_schmidt=3), dict(tile_fusion=2), dict(tile_fusion=3),
                                dict(cluster_cells=4096), dict(schur=3), dict(galerkin=2),
                                dict(galerkin=1, kcycle=2), dict(inner_cg=-1), dict(inner_cg=17), dict(res64=2)])
def test_options_outside_their_range_are_rejected_not_clamped(kw):
    """pyro_stokes_footprint (host logic, no GPU) answers 0 for an option outside its documented
    range, as pyro_stokes_create answers PYRO_E_INVALID; the same options in range are served."""
    import paper_2603_14040_b300 as P
    assert P.footprint(64, 64, P.default_opts()) > 0
    assert P.footprint(64, 64, P.default_opts(**kw)) == 0


def test_product_path_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_2603_14040_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
