"""The serving loop: continuous batching of decode requests of several codes.

Requests of four codes, with random frame counts and Eb/N0, are submitted
while others are decoding (from a client thread, with gaps), into pools too
small to hold them all at once, so admission waits for slots to free up.
Every request's outputs must equal those of the batched form run on that
request alone: each frame's arithmetic does not depend on the mix.
"""
import threading
import time

import numpy as np
import pytest

from workloads import awgn_frames, ebch

pytestmark = pytest.mark.gpu

CODES = ["ebch_32_26", "ebch_64_57", "ebch_64_51", "ebch_128_120"]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2310_10737_gb300 as sg
    return torch, sg


def _requests(n_req, seed, max_frames=24):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_req):
        ci = int(rng.integers(0, len(CODES)))
        code = ebch(CODES[ci])
        F = int(rng.integers(1, max_frames + 1))
        _, _, lch = awgn_frames(code, F, float(rng.uniform(2.5, 4.0)), seed=seed * 1000 + i)
        if i == 3:
            lch[0, 1, 1] = np.nan  # a request with an invalid frame
        out.append((ci, lch))
    return out


@pytest.mark.parametrize("epoch_halves", [1, 3])
def test_results_are_the_same_alone_and_in_the_mix(env, epoch_halves):
    torch, sg = env
    codes = [sg.Code.from_linear_code(ebch(nm)) for nm in CODES]
    reqs = _requests(40, 11 + epoch_halves)
    # each request alone, batched form
    alone = []
    for ci, lch in reqs:
        o = sg.product_decode(codes[ci], torch.from_numpy(lch).cuda(), L=4, query_cap=10**4, alpha=0.5,
                              max_iter=20, persistent=True)
        torch.cuda.synchronize()
        alone.append({k: v.cpu().numpy() for k, v in o.items() if hasattr(v, "cpu")})
    srv = sg.Server(codes, slots=[40, 40, 40, 30], L=4, query_cap=10**4, alpha=0.5, max_iter=20,
                    epoch_halves=epoch_halves)
    tickets = [None] * len(reqs)
    pinned = [torch.from_numpy(lch).pin_memory() for _, lch in reqs]

    def client():
        for i, (ci, _) in enumerate(reqs):
            tickets[i] = srv.submit(ci, pinned[i])
            if i % 5 == 4:
                time.sleep(0.002)  # arrivals while earlier requests decode

    th = threading.Thread(target=client)
    th.start()
    th.join()
    lat = []
    for i, (ticket, out) in enumerate(tickets):
        done, ms = srv.wait(ticket, timeout_ms=120000)
        assert done
        lat.append(ms)
        for key in ("bits", "half_iters", "status", "queries"):
            np.testing.assert_array_equal(out[key], alone[i][key], err_msg=f"request {i} {key}")
    st = srv.stats()
    assert st["requests_done"] == len(reqs) and st["frames_resident"] == 0 and st["requests_waiting"] == 0
    assert tickets[3][1]["status"][0] == 2
    assert all(x > 0 for x in lat)
    # a request larger than its pool can never be admitted; a ticket is reported once
    with pytest.raises(sg.SograndError):
        srv.submit(3, np.zeros((31, 128, 128), np.float32))
    with pytest.raises(sg.SograndError):
        srv.wait(tickets[0][0])
    srv.close()
    for c in codes:
        c.close()
