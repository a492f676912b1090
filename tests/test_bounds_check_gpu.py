"""The bounds-checked build of the library (build.build(checked=True), compiled
with -DFIRE_BOUNDS_CHECK): every global index the step kernels form is checked
against its buffer; a bad one sets a status bit, reported as FIRE_ERR_BOUNDS,
and is replaced by an index inside the buffer, so the kernel neither traps nor
touches memory outside it.

The test runs small cases through every step-kernel variant, both precisions,
the linear fuel-fraction scheme and the ensemble, in child processes: once on
the checked library and once on the normal one (tests/bounds_child.py). No
case may report FIRE_ERR_BOUNDS, and every state and heat grid must be the same
bits in both builds (the checks change no value). The checker itself is
tested on indices just inside and just outside a buffer, without using them
for an access."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def libs():
    import torch
    from paper_1102_1343_gb300 import build
    assert torch.cuda.is_available()
    return build.build(), build.build(checked=True)


def run_child(tmp_path, lib, name):
    env = dict(os.environ)
    env["WRFFIRE_LIBRARY"] = lib
    out = tmp_path / f"{name}.npz"
    p = subprocess.run([sys.executable, os.path.join(HERE, "bounds_child.py"), str(out)],
                       env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    return dict(np.load(out))


def test_checked_build_flags_no_index_and_changes_no_bit(libs, tmp_path):
    import paper_1102_1343_gb300 as pkg
    normal = run_child(tmp_path, libs[0], "normal")
    checked = run_child(tmp_path, libs[1], "checked")
    assert not bool(normal["checked"]) and bool(checked["checked"])
    assert set(normal) == set(checked)
    statuses = [k for k in checked if k.endswith("_status")]
    assert len(statuses) == 44  # 4 meshes x (6 FP32 + 4 FP64 kernels), 2 linear, 2 ensembles
    for k in statuses:
        assert int(checked[k]) != pkg.FIRE_ERR_BOUNDS, k
        assert int(checked[k]) == int(normal[k]), k
    for k in checked:
        if k == "checked" or k.endswith("_status"):
            continue
        assert np.array_equal(normal[k], checked[k]), k
    # the cases burn (not all ignition times still unset)
    assert all(np.isfinite(checked[k]).sum() > 0 for k in checked if k.endswith("_1"))


def test_index_check_flags_outside_indices(libs):
    """The check on the indices -1, 0, 9, 10 of a 10-element buffer, in a
    child process on the checked library (the normal one refuses the call)."""
    code = ("import sys; sys.path.insert(0, %r); import paper_1102_1343_gb300 as p; "
            "print(p.fire_bounds_selftest())" % ROOT)
    env = dict(os.environ)
    env["WRFFIRE_LIBRARY"] = libs[1]
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stderr[-3000:]
    assert p.stdout.strip().splitlines()[-1] == "[1, 0, 0, 1]"
    env["WRFFIRE_LIBRARY"] = libs[0]
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=300)
    assert p.returncode != 0 and "FireError" in p.stderr
