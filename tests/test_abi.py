"""The C-ABI library: it builds, loads without a GPU, exports every symbol the
header declares, and its parameter layout matches the oracle's block by block."""
import os
import re

import pytest

import oracle
from paper_2011_07125_gb300 import binding, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in ("ferminet.h", "ferminet_diag.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        names |= set(re.findall(r"\b(ferminet_\w+)\s*\(", src))
    return sorted(names)


def test_header_symbols_exported():
    lib = binding.load()
    names = _declared()
    assert len(names) >= 12
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(binding.EXPORTS) <= set(names)


@pytest.mark.parametrize("name", synth.WORKLOADS)
def test_layout_matches_oracle(name):
    net = synth.workload(name).net
    a = binding.net_layout(net)
    b = oracle.layout(net)
    assert [(e.name, e.offset, e.count, e.fan_in, e.kind) for e in a] == \
           [(e.name, e.offset, e.count, e.fan_in, e.kind) for e in b]


@pytest.mark.parametrize("shape", [(1, 4, 4, 1, 1, 0, 1), (3, 16, 8, 2, 2, 3, 2), (2, 32, 32, 4, 7, 7, 5),
                                   (1, 4, 4, 1, 1, 0, 1, 1), (2, 32, 32, 4, 7, 7, 5, 1)])
def test_layout_matches_oracle_odd_shapes(shape):
    """Odd shapes, with the isotropic and the full-covariance envelope."""
    net = synth.Net(*shape)
    a = binding.net_layout(net)
    b = oracle.layout(net)
    assert [(e.name, e.offset, e.count, e.fan_in, e.kind) for e in a] == \
           [(e.name, e.offset, e.count, e.fan_in, e.kind) for e in b]


def test_invalid_shape_rejected():
    with pytest.raises(binding.FermiNetError):
        binding.net_layout(synth.Net(0, 4, 4, 1, 1, 1, 1))
    with pytest.raises(binding.FermiNetError):
        binding.net_layout(synth.Net(1, 4, 4, 1, 1, 1, 1, envelope=2))
