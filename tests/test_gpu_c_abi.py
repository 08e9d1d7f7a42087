"""The library used from plain C (tests/c_abi_demo.c, compiled with the
system C compiler against include/klb.h and libklb.so, device buffer and
stream from the CUDA runtime): its observables equal, bit for bit, those of
the same lattice stepped through the Python binding."""
import glob
import os
import shutil
import subprocess

import pytest

from paper_2403_15768_gb300 import build, inputs, klb

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cudart_dir():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    for d in [os.path.join(cuda, "lib64"), *glob.glob(os.path.join(cuda, "targets", "*", "lib"))]:
        if os.path.exists(os.path.join(d, "libcudart.so")):
            return cuda, d
    pytest.skip("no libcudart.so")


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_c_caller_matches_python(tmp_path, storage):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    cuda, cudart = _cudart_dir()
    exe = tmp_path / "c_abi_demo"
    subprocess.run([cc, "-std=c11", "-O1", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                    os.path.join(ROOT, "tests", "c_abi_demo.c"), lib, "-L", cudart, "-lcudart",
                    "-Wl,-rpath," + os.path.dirname(lib) + ":" + cudart, "-o", str(exe)], check=True)
    w = inputs.PIPE_D3Q19_FP32.with_(nx=64, ny=24, nz=24, radius=8, shell=3, storage=storage,
                                     couplings=(0.05, 0.02, 0.1, 0.0, 0.01))
    steps = 50
    args = [str(v) for v in (w.nx, w.ny, w.nz, w.radius, w.shell, steps, w.tau[0], w.G[0], *w.couplings,
                             klb.STORAGE[storage])]
    r = subprocess.run([str(exe), *args], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    got = dict(line.split() for line in r.stdout.splitlines())
    lat = klb.lattice_from_workload(w)
    lat.step(steps)
    ob = lat.observables()
    assert int(got["step"]) == ob["step"] == steps
    for k in ("flow_rate", "slip_length", "u_slip", "residual"):
        assert float.fromhex(got[k]) == ob[k], k
    for s in range(3):
        assert float.fromhex(got[f"mean_u{s}"]) == ob["mean_u"][s]
        assert float.fromhex(got[f"mass{s}"]) == ob["mass"][s]
