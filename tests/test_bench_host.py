"""Host-side logic of bench.py (no GPU): the algorithmic byte count used for
the HBM view of the GEMM-class roofline, the key of the DRAM traffic record and
the launcher of several ranks."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_2011_07125_gb300 import synth  # noqa: E402


def _launch_bytes(net):
    """The same count, launch by launch: (rows, K read, N written) of every
    GEMM of the local-energy pass, plus the per-walker U term the layers read."""
    n, N = net.n_elec, net.n_nuc
    C = 3 * n + 2
    launches = []
    for l in range(net.n_layers):
        a1 = 4 * N if l == 0 else net.d1
        a2 = 4 if l == 0 else net.d2
        launches.append((C, 2 * a1, net.d1))                   # U = spin means x V_bc
        launches.append((n * C, a1 + 2 * a2, net.d1))          # layer: [h, pair means] x [V_a; V_de]
        launches.append((C, net.d1, 0))                        # U read by the layer
    launches.append((n * C, net.d1, 0))                        # orbitals read h^L
    same_spin = (net.n_up ** 2 + net.n_down ** 2) * net.n_det * C
    return 4 * (sum(r * (k + w) for r, k, w in launches) + same_spin)


@pytest.mark.parametrize("name", ["li", "ne", "ar", "c4h6"])
def test_gemm_class_bytes_match_launch_count(name):
    net = synth.workload(name).net
    assert bench.gemm_class_alg_bytes(net) == pytest.approx(_launch_bytes(net), rel=0, abs=0)


def test_gemm_class_bytes_c4h6_value():
    # 30 electrons, 92 real columns, 10 nuclei, d1 = 256, d2 = 32, 16 determinants
    assert bench.gemm_class_alg_bytes(synth.workload("c4h6").net) == 29257472


def test_source_key_ignores_comments_not_code():
    """The traffic record's source key: comment and layout edits keep it, a
    changed token does not."""
    src = b"int f(int x) {  // doubled\n  return 2 * x; /* no overflow\n check */\n}\n"
    same = b"int f(int x) {\n\n    return 2 * x;\n}"
    other = b"int f(int x) { return 3 * x; }"
    assert bench.code_only(src) == bench.code_only(same) == b"int f(int x) { return 2 * x; }"
    assert bench.code_only(src) != bench.code_only(other)
    assert len(bench.kernel_source_hash()) == 16


def test_layer_groups_compare_as_tiles():
    """The traffic record's layer_groups matches the tile the library selects:
    0 is the default tile (as many groups as fit 256 rows in multiples of 16)."""
    assert bench.layer_groups_used(0, 88) == bench.layer_groups_used(2, 88) == 2   # C4H4: 176-row tiles
    assert bench.layer_groups_used(0, 96) == 2 and bench.layer_groups_used(1, 96) == 1  # C4H6
    assert bench.layer_groups_used(0, 16) == 16 and bench.layer_groups_used(3, 16) == 3


def _bench(*args, env=None):
    import subprocess
    e = dict(os.environ)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        e.pop(k, None)
    e.update(env or {})
    return subprocess.run([sys.executable, bench.__file__, *args], capture_output=True, text=True, env=e,
                          timeout=300)


def test_gpus_flag_starts_that_many_ranks():
    """`bench.py --gpus 2` without a launcher starts two ranks itself (host
    ranks over gloo here), and rank 0 reports both."""
    import json
    r = _bench("--gpus", "2", "--check-launch")
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["n_gpus"] == 2 and line["ranks"] == [0, 1]


def test_gpus_flag_disagreeing_with_launcher_fails():
    r = _bench("--gpus", "2", "--check-launch", env={"WORLD_SIZE": "1", "RANK": "0"})
    assert r.returncode != 0
    assert "--gpus 2" in r.stderr
