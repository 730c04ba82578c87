"""The C ABI library (no GPU needed): it builds, loads, exports every entry point include/ksdf.h declares,
and validates parameters before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_29227_gb300 import build, ksdf

    build.build()
    return ksdf.load()


def declared(header="ksdf.h"):
    hdr = open(os.path.join(ROOT, "include", header)).read()
    return re.findall(r"^(?:ksdf_status|const char\*|int)\s+(ksdf_\w+)\(", hdr, re.M)


def test_exports_every_declared_symbol(lib):
    from paper_2603_29227_gb300 import ksdf

    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(ksdf.ABI_FUNCTIONS)


def test_exports_every_front_end_symbol(lib):
    """include/ksdf_bhm.h (the BHM front-end) is part of the same library and of its binding."""
    from paper_2603_29227_gb300 import bhm

    names = declared("ksdf_bhm.h")
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(bhm.BHM_ABI_FUNCTIONS)


def test_front_end_parameters_rejected_without_cuda(lib):
    from paper_2603_29227_gb300 import bhm, ksdf

    bhm.load()
    good = dict(bhm.DEFAULTS)
    bad = [dict(good, hinge_spacing=0.0), dict(good, block_hinges=3), dict(good, block_hinges=17),
           dict(good, gamma=-1.0), dict(good, phi_min=0.0), dict(good, phi_min=1.0), dict(good, prior_var=0.0),
           dict(good, em_iters=0), dict(good, em_iters=5), dict(good, xi_init=-1.0), dict(good, free_step=0.0),
           dict(good, free_gap=-0.1), dict(good, tau_alpha=0.0), dict(good, tau_alpha=1.5), dict(good, beta=0.0),
           dict(good, march_sub=3), dict(good, bias_feature=2), dict(good, gamma=1.0),  # window beyond 2 hinges
           dict(good, block_hinges=4)]  # 2 r + 1 > n_h
    for p in bad:
        h = ctypes.c_void_p()
        pr = bhm.make_params(p)
        assert lib.ksdf_bhm_create(ctypes.byref(pr), 100, 0, None, ctypes.byref(h)) == ksdf.KSDF_ERR_ARG, p
        assert not h.value
    pr = bhm.make_params(good)
    h = ctypes.c_void_p()
    assert lib.ksdf_bhm_create(ctypes.byref(pr), 0, 0, None, ctypes.byref(h)) == ksdf.KSDF_ERR_ARG
    assert lib.ksdf_bhm_destroy(None) == ksdf.KSDF_OK
    assert lib.ksdf_bhm_sync_status(None) == ksdf.KSDF_ERR_ARG
    assert lib.ksdf_bhm_update(None, None, None, 0) == ksdf.KSDF_ERR_ARG


def test_invalid_parameters_rejected_without_cuda(lib):
    from paper_2603_29227_gb300 import ksdf

    good = dict(dim=3, origin=(0, 0, 0), cell=0.5, margin=0.1, n_max=256, k_cand=8, softmin_alpha=0.0, sign_mode=0,
                **{"lambda": 300.0})
    bad = [dict(good, dim=4), dict(good, cell=0.0), dict(good, margin=-1.0), dict(good, n_max=0),
           dict(good, n_max=513), dict(good, k_cand=0), dict(good, k_cand=33), dict(good, **{"lambda": -1.0}),
           dict(good, sign_mode=2), dict(good, margin=10.0), dict(good, kernel=2), dict(good, kernel=-1)]
    for p in bad:
        h = ctypes.c_void_p()
        pr = ksdf.make_params(p)
        assert lib.ksdf_create(ctypes.byref(pr), None, ctypes.byref(h)) == ksdf.KSDF_ERR_ARG, p
        assert not h.value
    # NULL handles are rejected everywhere
    assert lib.ksdf_destroy(None) == ksdf.KSDF_ERR_ARG
    assert lib.ksdf_sync_status(None) == ksdf.KSDF_ERR_ARG
    assert lib.ksdf_fit(None, None, None, None, 1) == ksdf.KSDF_ERR_ARG


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2603_29227_gb300 import ksdf

    saved = ksdf._lib
    ksdf._lib = None
    try:
        with pytest.raises(RuntimeError):
            ksdf.load(str(tmp_path / "missing.so"))
    finally:
        ksdf._lib = saved


def test_graft_entry_build_importable():
    import __graft_entry__

    assert callable(__graft_entry__.build) and callable(__graft_entry__.smoke)


def test_peaks_library_exports_its_header():
    """The benchmark's probe library (include/ksdf_peaks.h) builds beside libksdf.so and exports what its
    header declares; libksdf.so itself does not carry the probes."""
    import ctypes as ct

    from paper_2603_29227_gb300 import build, ksdf, peaks

    build.build()
    hdr = open(os.path.join(ROOT, "include", "ksdf_peaks.h")).read()
    names = re.findall(r"^(?:int|const char\*)\s+(ksdf_peaks_\w+)\(", hdr, re.M)
    assert sorted(names) == ["ksdf_peaks_last_error", "ksdf_peaks_measure"]
    lib = peaks.load()
    for n in names:
        assert hasattr(lib, n), n
    main = ct.CDLL(ksdf.LIB_PATH)
    assert not hasattr(main, "ksdf_peaks_measure")
    # a NULL output pointer is rejected before any CUDA call
    assert lib.ksdf_peaks_measure(0, None, None) == 1
