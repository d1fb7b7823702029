"""Host-side logic of bench.py (no GPU): the algorithmic byte count used for
the HBM view of the GEMM-class roofline."""
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
