"""The C-ABI library builds, loads and exports every function its header declares.
These tests make no compute call and need no GPU."""
import ctypes
import subprocess

import pytest

from paper_1310_4374_gb300 import binding as B
from paper_1310_4374_gb300 import build as _build


def test_header_declares_the_boundary():
    names = B.header_functions()
    for required in ("psum_plan_create", "psum_plan_create_ex", "psum_eval", "psum_eval_host", "psum_sync",
                     "psum_get_coeffs", "psum_plan_info", "psum_destroy", "psum_strerror", "psum_opts_default",
                     "psum_profile", "psum_last_timings"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = _build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in B.header_functions() if n not in exported]
    assert not missing, missing
    lib = B.load()
    for n in B.header_functions():
        assert hasattr(lib, n)


def test_strerror_and_defaults_without_gpu():
    assert B.psum_strerror(B.PSUM_OK) == "ok"
    for s in range(1, 11):
        assert B.psum_strerror(s) and B.psum_strerror(s) != "unknown status"
    assert B.psum_strerror(99) == "unknown status"
    o = B.psum_opts_default()
    assert tuple(o.d) == (1.0, 1.0, 1.0) and o.p == 8 and o.M == 200 and tuple(o.K) == (1, 1, 1)
    assert o.precision == B.PSUM_FP64 and o.mean_mode == B.PSUM_MEAN_ZERO
    assert o.pair_kernel == B.PAIR_KERNELS["auto"] == 0
    assert o.check_form == B.CHECK_FORMS["auto"] == 0


@pytest.mark.parametrize("d,p,M,prec,K", [
    ((1, 1, 1), 0, 200, "fp64", (1, 1, 1)),        # p < 1
    ((1, 1, 1), 41, 5000, "fp64", (1, 1, 1)),      # p above the supported maximum
    ((1, 1, 1), 8, 79, "fp64", (1, 1, 1)),         # M < P - 1 (rank condition)
    ((1, -1, 1), 8, 200, "fp64", (1, 1, 1)),       # d <= 0
    ((1, 1, float("nan")), 8, 200, "fp64", (1, 1, 1)),
    ((1, 1, 1), 8, 200, 7, (1, 1, 1)),             # unknown precision
    ((1, 1, 1), 8, 200, 3, (1, 1, 1)),
    ((1, 1, 1), 8, 200, "fp64", (1, 4, 1)),        # K out of range
])
def test_invalid_plan_arguments_are_rejected_on_the_host(d, p, M, prec, K):
    with pytest.raises(B.PsumError) as e:
        B.psum_plan_create_ex(d, p, M, prec, "zero", K)
    assert e.value.status == B.PSUM_ERR_ARG


def test_null_arguments_are_rejected():
    lib = B.load()
    assert lib.psum_plan_create_ex(None, None) == B.PSUM_ERR_ARG
    assert lib.psum_eval(None, 10, None, None, None, None, None) == B.PSUM_ERR_ARG
    assert lib.psum_sync(None, None) == B.PSUM_ERR_ARG
    assert lib.psum_plan_info(None, None) == B.PSUM_ERR_ARG
    k = ctypes.c_int(-1)
    assert lib.psum_pair_kernel(None, 10, ctypes.byref(k), None) == B.PSUM_ERR_ARG
    assert lib.psum_check_form(None, ctypes.byref(k)) == B.PSUM_ERR_ARG
    lib.psum_destroy(None)
    h = ctypes.c_void_p()
    assert lib.psum_plan_create(1.0, 1.0, 1.0, 8, 10, ctypes.byref(h)) == B.PSUM_ERR_ARG


@pytest.mark.parametrize("lam", [0.5, 1.0, -1.0, 9.0, float("nan")])
def test_ball_radius_out_of_range_is_rejected(lam):
    # lambda = Rb/R0 must exceed 1 (the ball holds the box) and stay within the image table
    with pytest.raises(B.PsumError) as e:
        B.psum_plan_create_ex((1, 1, 1), 8, 200, lam=lam)
    assert e.value.status == B.PSUM_ERR_ARG


@pytest.mark.parametrize("kw", [dict(n_rbf=300), dict(n_rbf=-1), dict(n_rbf=5000), dict(rbf_radius=0.9),
                                dict(rbf_radius=float("inf")), dict(basis=2)])
def test_rbf_options_out_of_range_are_rejected(kw):
    # Eq. 5 needs the centres outside the circumsphere, and M >= n_rbf check points
    args = dict(basis="rbf", n_rbf=100)
    args.update(kw)
    with pytest.raises(B.PsumError) as e:
        B.psum_plan_create_ex((1, 1, 1), 8, 200, **args)
    assert e.value.status == B.PSUM_ERR_ARG


def test_gauss_grid_fixes_the_number_of_check_points():
    with pytest.raises(B.PsumError) as e:
        B.psum_plan_create_ex((1, 1, 1), 8, 5, points="gauss")      # M must be 0 or (p+1)(2p+1)
    assert e.value.status == B.PSUM_ERR_ARG
    with pytest.raises(B.PsumError) as e:
        B.psum_plan_create_ex((1, 1, 1), 8, 200, points=7)
    assert e.value.status == B.PSUM_ERR_ARG


@pytest.mark.parametrize("pair_kernel", [-1, 3, 99])
def test_unknown_pair_kernel_is_rejected(pair_kernel):
    # checked on the host before any device call
    o = B.psum_opts_default()
    o.p, o.M = 8, 200
    o.pair_kernel = pair_kernel
    h = ctypes.c_void_p()
    assert B.load().psum_plan_create_ex(ctypes.byref(o), ctypes.byref(h)) == B.PSUM_ERR_ARG


@pytest.mark.parametrize("check_form,prec,lam", [(-1, "fp32c", 0.0), (3, "fp64", 0.0),
                                                 (2, "fp32c", 1.5),      # layers: block near sets only,
                                                 (2, "fp64", 1.7)])      # not the ball
def test_invalid_check_form_is_rejected(check_form, prec, lam):
    # checked on the host before any device call
    o = B.psum_opts_default()
    o.p, o.M = 8, 200
    o.precision = B.PRECISIONS[prec]
    o.lambda_ = lam
    o.check_form = check_form
    h = ctypes.c_void_p()
    assert B.load().psum_plan_create_ex(ctypes.byref(o), ctypes.byref(h)) == B.PSUM_ERR_ARG


def test_plan_files_that_do_not_match_are_refused_on_the_host(tmp_path):
    # psum_plan_load checks the file before any device call: a missing file, a wrong magic word,
    # a truncated file and a bad checksum are PSUM_ERR_IO
    with pytest.raises(B.PsumError) as e:
        B.psum_plan_load(tmp_path / "missing.plan")
    assert e.value.status == B.PSUM_ERR_IO
    bad = tmp_path / "bad.plan"
    bad.write_bytes(b"NOTAPLAN" + bytes(200))
    with pytest.raises(B.PsumError) as e:
        B.psum_plan_load(bad)
    assert e.value.status == B.PSUM_ERR_IO
    # a well-formed header with a pseudo-inverse of 4 doubles but a wrong checksum
    o = B.psum_opts_default()
    body = (b"PSUMPLN1" + ctypes.sizeof(o).to_bytes(4, "little") + bytes(o) + bytes(8) + (7).to_bytes(4, "little")
            + bytes(8) + (4).to_bytes(8, "little") + bytes(32))
    for blob in (body + (12345).to_bytes(8, "little"), body[:-5]):
        bad.write_bytes(blob)
        with pytest.raises(B.PsumError) as e:
            B.psum_plan_load(bad)
        assert e.value.status == B.PSUM_ERR_IO
    with pytest.raises(B.PsumError) as e:
        B.psum_plan_save(None, tmp_path / "x.plan")
    assert e.value.status == B.PSUM_ERR_ARG
