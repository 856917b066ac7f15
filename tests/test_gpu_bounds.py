"""The debug build with range-checked kernel indices (libspinsim_bounds.so,
compiled with -DSPINSIM_BOUNDS).

A child process loads the debug library (SPINSIM_BOUNDS=1) and runs the edge
cases of one batch (K = 0, K = 1, L = 1, L = 3, ragged tails, invalid
requests, both spins), chain trees of every height, FP32-bulk and FP64, the
serving queue and the allocation-free entry point; then it reads the device
error words.  Every checked index must have stayed in range (word 0), and the
results must equal those of the normal library bit for bit: the checks skip
only out-of-range accesses and change no arithmetic.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
from paper_2204_05586_gb300 import spinsim as S, workloads as W

def cases():
    base = W.field(bias_hz=150e3, drive_x_hz=4e3, drive_hz=150.5e3, quad_hz=300.0, pulses=[(90.0, 3e-4, 1e-4)])
    edge = [W.request(2, base, 0.0, 0.0, 1e-8, 1e-6), W.request(2, base, 0.0, 1e-6, 1e-8, 1e-6),
            W.request(1, base, 0.0, 7e-6, 1e-6, 1e-6), W.request(2, base, 2e-5, 2e-5 + 529e-6, 1e-7, 1e-6),
            W.request(1, base, 0.0, 1037e-6, 2.5e-7, 1e-6), W.request(2, base, 0.0, 3e-6, 1e-6 / 3, 1e-6),
            W.request(2, base, 0.0, 1e-5, 3e-7, 1e-6),
            W.request(2, base, 0.0, 1e-5, 1e-8, 1e-6, psi0=[1.0, 0.5, 0.0])]
    tall = [W.request(2, base, 0.0, K * 1e-6, 1e-6, 1e-6) for K in (128, 129, 4097, 140000)]
    return edge, tall + W.sweep(24, t_min=1e-4, t_max=3e-3)

out = {}
edge, batch = cases()
for prec in (S.PREC_FP64, S.PREC_FP32_BULK):
    with S.Simulator(precision=prec) as sim:
        res_e = sim.simulate(edge[:6], check=False)
        res_b = sim.simulate(batch)
        bad = sim.simulate(edge[6:], check=False)
        out[f"edge{prec}"] = [o["states"].cpu().numpy().tolist() for o in res_e]
        out[f"batch{prec}"] = [np.asarray(o["states"].cpu().numpy()[::97]).tolist() for o in res_b]
        out[f"bad{prec}"] = [o["status"] for o in bad]
with S.Simulator(precision=S.PREC_FP32_BULK) as sim:
    outs = sim.allocate(batch[4:10])
    res = sim.results_struct(outs)
    for q, r in zip(batch[4:10], res):
        st, t = S.spinsim_submit(sim.handle, S.make_request(q), r)
        assert S.spinsim_poll(sim.handle, t, 20_000_000) == S.OK
    out["served"] = [torch.view_as_complex(o["states"][:o["K"]]).cpu().numpy()[::31].tolist() for o in outs]
q = W.spin_one_sensing(t_end=3e-3)
K = S.spinsim_counts(S.make_request(q))[1]
st_buf = torch.empty((K, 3, 2), dtype=torch.float64, device="cuda")
r = S.spinsim_result(); r.states = st_buf.data_ptr(); r.capacity = K
assert S.spinsim_simulate_static(S.make_config(), S.make_request(q), r, 0) == S.OK
torch.cuda.synchronize()
out["static"] = torch.view_as_complex(st_buf).cpu().numpy()[::17].tolist()
out["word"] = list(S.spinsim_debug_bounds(0))
print("RESULT " + json.dumps(out, default=lambda z: [z.real, z.imag]))
'''


def run_child(bounds: bool):
    env = dict(os.environ, SPINSIM_BOUNDS="1" if bounds else "0")
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_every_checked_index_stays_in_range_and_results_are_unchanged():
    dbg = run_child(True)
    assert dbg["word"] == [0, 0], f"out-of-range kernel indices: word {dbg['word'][1]:#x}"
    ref = run_child(False)
    assert ref["word"][0] == -8                     # the normal library has no checks (E_UNSUPPORTED)
    for key in ref:
        if key != "word":
            assert dbg[key] == ref[key], key
    assert dbg["bad0"] == [-2, -3] and dbg["bad1"] == [-2, -3]
