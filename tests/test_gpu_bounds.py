"""The debug build with index checks (-DKLB_BOUNDS=1, klb_bounds_status)
finds no out-of-range index on any lattice kind, storage, geometry, batch or
noise path exercised here.  It runs in a child process that loads the debug
library (the normal one stays loaded in this process)."""
import os
import subprocess
import sys
import textwrap

import pytest

from paper_2403_15768_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import torch
    from paper_2403_15768_gb300 import inputs, klb

    lib = klb.load_library()
    assert lib.klb_bounds_checked() == 1
    pipe = inputs.PIPE_D3Q19_FP32.with_(nx=37, ny=17, nz=15, radius=5, shell=2)
    cases = [
        pipe, pipe.with_(storage="fp64"), pipe.with_(storage="fp16"), pipe.with_(storage="bf16"),
        pipe.with_(nx=1), pipe.with_(nx=64, ny=12, nz=12, radius=3, shell=1),
        pipe.with_(iface_bc="bounceback"),
        inputs.SLAB_D2Q9_FP64.with_(nx=33), inputs.SLAB_D2Q9_FP64.with_(nx=33, storage="fp16"),
        pipe.with_(geom="slab", nx=70, ny=14, nz=3, width=6, shell=3),
    ]
    lats = []
    for k, w in enumerate(cases):
        lat = klb.lattice_from_workload(w)
        d, u = inputs.perturbation(w, k, 1e-3)
        lat.init_equilibrium(d, u)
        lat.step(70)  # past two reference refreshes of 16-bit storage
        lat.observables()
        lat.get_field()
        lat.get_state()
        lats.append(lat)
    batch = klb.Batch([l for l in lats if l.desc.storage == 1][:3])
    batch.step(13)
    noisy = klb.lattice_from_workload(pipe)
    noisy.set_fluctuations(1e-5, 3)
    noisy.step(9)
    lats.append(noisy)
    bad = [(c, l.bounds_status()) for c, l in zip(cases + ["noise"], lats)]
    bad = [b for b in bad if b[1]]
    print("OK" if not bad else "BAD %r" % bad)
""")


def test_debug_build_has_no_out_of_range_index():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = build.build(bounds=True)
    env = dict(os.environ, KLB_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().splitlines()[-1] == "OK", r.stdout + r.stderr
