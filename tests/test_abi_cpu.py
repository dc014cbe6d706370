"""CPU checks of the C ABI: the library builds for sm_103a, loads without a
GPU, and exports every entry point include/qcl.h declares.  Argument
validation that happens before any CUDA call is exercised too."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2608_14544_gb300 import build, qcl

    build.build()
    return qcl.load()


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(qcl_\w+)\s*\(", txt, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    from paper_2608_14544_gb300 import qcl

    declared = _declared()
    assert len(declared) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", qcl.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(qcl_\w+)", out))
    assert declared <= exported, declared - exported
    assert set(qcl.EXPORTS) == declared
    for name in declared:
        assert hasattr(lib, name)


def test_library_targets_sm_103a(lib):
    from paper_2608_14544_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_model_validation_without_gpu(lib):
    from paper_2608_14544_gb300 import qcl

    def desc(ns, n, E, K, mass=None, omega=None, hbar=1.0, pmax=0.5, rep=0, reserved=0, hop=1.0):
        arrs = [np.ones(n) if mass is None else np.asarray(mass, float),
                np.ones(n) if omega is None else np.asarray(omega, float),
                np.ascontiguousarray(E, dtype=float), np.ascontiguousarray(K, dtype=float)]
        d = qcl.ModelDesc(ns, n, hbar, *[a.ctypes.data for a in arrs], hop, pmax, rep, reserved)
        return d, arrs

    h = C.c_void_p()
    E = np.array([[0.0, 0.5], [0.5, 0.0]])
    K = np.array([[[1.0, 0.0], [0.0, -1.0]]])
    d, keep = desc(1, 1, E, K)
    assert lib.qcl_create_model(C.byref(d), C.byref(h)) == 1 and not h.value
    d, keep = desc(2, 1, np.array([[0.0, 0.5], [0.4, 0.0]]), K)
    assert lib.qcl_create_model(C.byref(d), C.byref(h)) == 1
    assert b"symmetric" in lib.qcl_last_error()
    d, keep = desc(2, 1, E, K, mass=[-1.0])
    assert lib.qcl_create_model(C.byref(d), C.byref(h)) == 1
    d, keep = desc(2, 1, E, K, pmax=1.5)
    assert lib.qcl_create_model(C.byref(d), C.byref(h)) == 1
    # transition-probability shape: a step's weight factor stays within
    # [2^-16, 2^17] where the model fixes it (stay 1/(1 - p), hop 1/kappa .. 2/kappa)
    for hop, pmax in ((2.0 ** -17, 0.5), (2.0 ** 17, 0.5), (-1.0, 0.5), (float("nan"), 0.5),
                      (1.0, 1.0 - 2.0 ** -17), (1.0, 1.0), (1.0, -0.1)):
        d, keep = desc(2, 1, E, K, pmax=pmax, hop=hop)
        assert lib.qcl_create_model(C.byref(d), C.byref(h)) == 1 and not h.value, (hop, pmax)
        assert b"hop_scale" in lib.qcl_last_error() or b"p_max" in lib.qcl_last_error()
    d, keep = desc(9, 1, np.eye(9), np.zeros((1, 9, 9)))
    assert lib.qcl_create_model(C.byref(d), C.byref(h)) == 2
    assert lib.qcl_create_model(None, C.byref(h)) == 1
    assert lib.qcl_destroy_model(None) == 0
    # representation: unknown code, diabatic beyond two states, reserved field
    d, keep = desc(2, 1, E, K, rep=5)
    assert lib.qcl_create_model(C.byref(d), C.byref(h)) == 1
    assert b"representation" in lib.qcl_last_error() or b"repr" in lib.qcl_last_error()
    # the diabatic representation takes any N_s: validation passes, and without
    # a GPU the call fails only at the device allocation
    d, keep = desc(3, 1, np.eye(3), np.zeros((1, 3, 3)), rep=qcl.REPR_DIABATIC)
    assert lib.qcl_create_model(C.byref(d), C.byref(h)) == 4 and not h.value
    assert b"cudaMalloc" in lib.qcl_last_error()
    d, keep = desc(2, 1, E, K, reserved=1)
    assert lib.qcl_create_model(C.byref(d), C.byref(h)) == 1


def test_option_and_null_checks_without_gpu(lib):
    from paper_2608_14544_gb300 import qcl

    assert lib.qcl_set_option(99, 0) == 1
    assert lib.qcl_set_option(1, -1) == 1
    assert lib.qcl_set_option(1, 0) == 0
    # where the N_s-state FP32 kernels keep the modes: 0, 1 or 2
    assert lib.qcl_set_option(qcl.OPT_MODES_IN_MEMORY, 3) == 1
    assert lib.qcl_set_option(qcl.OPT_MODES_IN_MEMORY, -1) == 1
    for v in (1, 2, 0):
        assert lib.qcl_set_option(qcl.OPT_MODES_IN_MEMORY, v) == 0
    assert lib.qcl_launch_count(None, 0) == 1
    c = C.c_int64()
    assert lib.qcl_launch_count(C.byref(c), 0) == 0
    assert lib.qcl_kernel_time(7, None, None) == 1
    b = C.c_size_t()
    assert lib.qcl_ensemble_bytes(None, None, C.byref(b)) == 1
    # a NULL model is rejected before any device work
    assert lib.qcl_finalize_observables(None, None, None, C.c_size_t(0), C.c_int64(1),
                                        C.c_int64(0), C.c_int64(1), None, C.c_size_t(0),
                                        None) == 1


def test_server_validation_without_gpu(lib):
    from paper_2608_14544_gb300 import qcl

    h = C.c_void_p()
    d = qcl.ServerDesc(None, 1 << 30, 4, 100, 1, 0, 0.0)
    assert lib.qcl_server_create(C.byref(d), C.byref(h)) == 1 and not h.value
    d = qcl.ServerDesc(256, 1024, 4, 100, 1, 0, 0.0)
    assert lib.qcl_server_create(C.byref(d), C.byref(h)) == 3
    # a negative or non-finite round work budget is rejected before any CUDA call
    for bad in (-1.0, float("nan"), float("inf")):
        d = qcl.ServerDesc(256, 1 << 30, 4, 100, 1, 0, 0.0, bad)
        assert lib.qcl_server_create(C.byref(d), C.byref(h)) == 1 and not h.value
        assert "round_flops" in qcl.last_error()
    assert lib.qcl_server_create(None, C.byref(h)) == 1
    assert lib.qcl_server_destroy(None) == 0
    st = C.c_int32()
    assert lib.qcl_server_poll(None, 1, C.byref(st), None, 0, None) == 1


def test_launch_shape_validation_without_gpu(lib):
    from paper_2608_14544_gb300 import qcl

    sh = qcl.LaunchShape(1, 0, 0.0)
    assert lib.qcl_set_launch_shape(None, C.byref(sh)) == 1
    assert lib.qcl_get_launch_shape(None, C.byref(sh)) == 1
    b = C.c_size_t()
    assert lib.qcl_autotune_bytes(None, 1024, 10, 10, C.byref(b)) == 1
    assert lib.qcl_autotune(None, 1024, 10, 0.01, 10, None, 0, C.byref(sh), None) == 1


def test_measure_peak_validation_without_gpu(lib):
    v = C.c_double()
    assert lib.qcl_measure_peak(0, None, None) == 1
    assert lib.qcl_measure_peak(7, C.byref(v), None) == 1


def test_product_path_fails_loudly_without_the_cuda_library_or_device():
    # no CPU fallback: a missing library is an ImportError, and without a GPU
    # the first call that needs device memory raises with the CUDA message
    import subprocess
    import sys

    code = (
        "from paper_2608_14544_gb300 import qcl, workloads as wl\n"
        "try:\n"
        "    qcl.load('/nonexistent/libqcl.so')\n"
        "    print('LOADED')\n"
        "except ImportError as e:\n"
        "    print('IMPORT-ERROR', 'no CPU fallback' in str(e))\n"
        "import torch\n"
        "if not torch.cuda.is_available():\n"
        "    try:\n"
        "        qcl.Model(wl.config(2)['model'])\n"
        "        print('MODEL')\n"
        "    except qcl.QclError as e:\n"
        "        print('QCL-ERROR', 'CUDA' in str(e))\n")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         timeout=300, cwd=os.path.dirname(os.path.dirname(__file__)))
    assert out.returncode == 0, out.stderr[-2000:]
    assert "IMPORT-ERROR True" in out.stdout
    assert "LOADED" not in out.stdout and "MODEL" not in out.stdout.split()
    assert "QCL-ERROR False" not in out.stdout
