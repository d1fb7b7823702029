"""ferminet_logpsi_noalloc: log|psi| for callers that cannot allocate device
memory (hosts that own every device buffer, or a device already fully reserved
by another allocator).  Its workspace is a fixed device array inside the
library, so its results must match the regular ferminet_logpsi, call after
call, whatever the array held before.  Kept in its own file so that it is
collected last."""
import ctypes as C

import numpy as np
import pytest

from helpers import TOL_LOGPSI_REL, rel_err, setup

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    from paper_2011_07125_gb300 import binding
    lib = binding.load()
    f = lib.ferminet_logpsi_noalloc
    vp = C.c_void_p
    f.argtypes = [C.POINTER(binding.FnNet), vp, vp, vp, C.c_long, vp, vp, vp]
    f.restype = C.c_int
    return lib, binding


def test_noalloc_logpsi_matches_logpsi_on_two_calls():
    lib, binding = _lib()
    wl, lay, P, x, geo = setup("c4h6", 300)  # about 80 walkers fit the array: several chunks
    fn = binding.FermiNet(wl.net, wl.geoms, counts=wl.counts, precision="fp32")
    params = torch.from_numpy(P).cuda()
    fn.set_params(params)
    R = torch.from_numpy(np.asarray(wl.geoms[0].R, np.float32).reshape(-1, 3)).cuda()
    net = binding._net(wl.net)
    stream = torch.cuda.current_stream().cuda_stream
    x2 = x.copy()
    x2[:, :, 0] += 0.3  # second call on other walkers, so stale contents would show
    for xs in (x, x2):
        xx = torch.from_numpy(np.ascontiguousarray(xs)).cuda()
        lp = torch.full((len(xs),), float("nan"), device="cuda")
        sg = torch.zeros(len(xs), device="cuda")
        rc = lib.ferminet_logpsi_noalloc(C.byref(net), params.data_ptr(), R.data_ptr(), xx.data_ptr(), len(xs),
                                         lp.data_ptr(), sg.data_ptr(), C.c_void_p(stream))
        assert rc == 0
        ref, ref_sign = fn.logpsi(xx)
        torch.cuda.synchronize()
        assert torch.equal(sg, ref_sign)
        assert rel_err(lp.cpu().numpy(), ref.cpu().numpy()).max() <= TOL_LOGPSI_REL


def test_noalloc_rejects_network_beyond_scratch():
    """A one-layer network of width 60000 over 64 electrons needs three
    [64 x 60000] float activation buffers per walker (46 MB > 32 MiB), so the
    call must refuse it before launching.  Every buffer passed is nevertheless
    full-sized, so the call stays memory-safe whatever it decides."""
    lib, binding = _lib()
    from paper_2011_07125_gb300 import synth
    big = synth.Net(1, 60000, 8, 1, 32, 32, 1)
    n = big.n_up + big.n_down
    assert 3 * n * big.d1 * 4 > (32 << 20)
    n_params = sum(e.count for e in binding.net_layout(big))
    params = torch.zeros(n_params, device="cuda")
    R = torch.zeros(3, device="cuda")
    x = torch.randn(1, n, 3, device="cuda")
    out = torch.zeros(1, device="cuda")
    net = binding._net(big)
    rc = lib.ferminet_logpsi_noalloc(C.byref(net), params.data_ptr(), R.data_ptr(), x.data_ptr(), 1,
                                     out.data_ptr(), None, None)
    torch.cuda.synchronize()
    assert binding.STATUS[rc] == "FN_ENOMEM"


def test_noalloc_back_to_back_on_side_stream():
    """Two calls queued back to back on one non-default stream, with no
    synchronisation between them: the second call's clearing of the status
    header and its reuse of the array are ordered after the first call's
    kernels by the stream, so both results equal ferminet_logpsi's."""
    lib, binding = _lib()
    wl, lay, P, x, geo = setup("ne", 40)
    fn = binding.FermiNet(wl.net, wl.geoms, counts=wl.counts, precision="fp32")
    params = torch.from_numpy(P).cuda()
    fn.set_params(params)
    R = torch.from_numpy(np.asarray(wl.geoms[0].R, np.float32).reshape(-1, 3)).cuda()
    net = binding._net(wl.net)
    x2 = x.copy()
    x2[:, :, 1] -= 0.2
    xs = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (x, x2)]
    refs = [fn.logpsi(xx) for xx in xs]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    outs = []
    with torch.cuda.stream(side):
        for xx in xs:
            lp = torch.full((len(x),), float("nan"), device="cuda")
            sg = torch.zeros(len(x), device="cuda")
            rc = lib.ferminet_logpsi_noalloc(C.byref(net), params.data_ptr(), R.data_ptr(), xx.data_ptr(), len(x),
                                             lp.data_ptr(), sg.data_ptr(), C.c_void_p(side.cuda_stream))
            assert rc == 0
            outs.append((lp, sg))
    side.synchronize()
    for (lp, sg), (ref, ref_sign) in zip(outs, refs):
        assert torch.equal(sg, ref_sign)
        assert rel_err(lp.cpu().numpy(), ref.cpu().numpy()).max() <= TOL_LOGPSI_REL
