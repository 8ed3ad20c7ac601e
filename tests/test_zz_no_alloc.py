"""The allocation-free self-energy entry point, called through the C ABI.

gkba_sigma_noalloc serves callers that cannot allocate device memory (code
running while a CUDA graph is captured, host frameworks that own every device
allocation, fixed memory budgets): its scratch is a static device array.  This
test checks it against the context-based gkba_sigma on two calls in a row,
with different inputs and sizes, so a result that leaned on the previous
call's leftovers in the shared scratch would fail.  The file sorts last so a
run that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import gkba_inputs as gi
import oracle as O
from _check import check

pytestmark = pytest.mark.gpu

TOL64 = 1e-10  # the FP64 path's tolerance in tests/test_gpu_parity.py




def test_noalloc_sigma_matches_gkba_sigma_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_01180_gb300 import build as b
    b.build()
    import paper_1905_01180_gb300 as P
    from paper_1905_01180_gb300 import gkba
    lib = gkba.load()
    stream = torch.cuda.current_stream()
    for call, (N, U, seed) in enumerate([(24, 3, 11), (9, 4, 12)]):
        s = gi.system(N, 8, seed=seed)
        G = np.stack([gi.random_pair(N, seed=100 * seed + u)[0] for u in range(U)])
        Gb = np.stack([gi.random_pair(N, seed=100 * seed + u)[1] for u in range(U)])
        with P.Context(s["h"], s["v"], s["d"], s["rho0"], 0.05) as ctx:
            ref = ctx.sigma(G, Gb)
        v_d = torch.from_numpy(s["v"]).cuda()
        G_d = torch.from_numpy(G).cuda()
        Gb_d = torch.from_numpy(Gb).cuda()
        S_d = torch.full_like(G_d, complex(np.nan, np.nan))
        msg = ctypes.create_string_buffer(256)
        st = lib.gkba_sigma_noalloc(N, U, v_d.data_ptr(), G_d.data_ptr(), Gb_d.data_ptr(),
                                    S_d.data_ptr(), stream.cuda_stream, msg, 256)
        stream.synchronize()
        assert st == gkba.OK, msg.value.decode()
        S = S_d.cpu().numpy()
        # against the context entry point, and against the oracle's Eq. (2b-opt) route
        oracle_ref = O.sigma_paper(s["v"], G, Gb)
        for u in range(U):
            check(S[u], ref[u], TOL64, f"call {call} unit {u} vs gkba_sigma")
            check(S[u], oracle_ref[u], TOL64, f"call {call} unit {u} vs oracle")


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1905_01180_gb300 import gkba
    lib = gkba.load()
    msg = ctypes.create_string_buffer(256)
    st = lib.gkba_sigma_noalloc(25, 1, None, None, None, None, None, msg, 256)
    assert st == gkba.EINVAL
    assert b"N=25" in msg.value
