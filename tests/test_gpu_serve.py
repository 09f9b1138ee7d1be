"""Serving: continuous batching of mixed requests, admission, cancellation,
injected allocation failure and head-of-line independence.

Faults are made on the host (an injected allocation failure, a request
cancelled while queued, oversize and queue-full rejections); nothing here
faults or hangs the GPU.
"""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

DUV = dict(wavelength_nm=193.0, na=1.35, n_medium=1.44, kind="annular", src_grid=21, sigma_in=0.6, sigma_out=0.9)
EUV = dict(wavelength_nm=13.5, na=0.33, n_medium=1.0, kind="annular", src_grid=21, sigma_in=0.6, sigma_out=0.9)


def _wait_all(srv, L, tickets, timeout_s=300):
    order, status = [], {}
    t0 = time.time()
    while len(status) < len(tickets) and time.time() - t0 < timeout_s:
        for t in tickets:
            if t in status:
                continue
            st = srv.poll(t, 0)
            if st != L.ETIMEOUT:
                status[t] = st
                order.append(t)
        time.sleep(0.002)
    return status, order


def _request_set(seed):
    st = synth.Stream(seed)
    reqs = []
    for i in range(20):
        n = int([256, 512, 1024][st.integers(0, 2, 1)[0]])
        euv = bool(st.integers(0, 1, 1)[0])
        k = int([8, 16][st.integers(0, 1, 1)[0]])
        kind = "image" if i % 2 == 0 else "ilt"
        prec = ["fft32", "fp16x3"][st.integers(0, 1, 1)[0]] if kind == "image" else "fft32"
        pixel = 1.0 if euv else 8.0
        if kind == "image":
            inp = synth.random_rect_mask(n, seed=seed * 100 + i, count=n // 4)
            tgt = None
        else:
            inp, tgt = synth.ilt_clip(n, pixel, seed=seed * 100 + i)
        reqs.append(dict(kind=kind, optics=EUV if euv else DUV, n=n, pixel=pixel, k=k, precision=prec,
                         input=np.ascontiguousarray(inp, dtype=np.float32),
                         target=None if tgt is None else np.ascontiguousarray(tgt, dtype=np.float32)))
    return reqs


def test_mixed_stream_matches_standalone(litho_lib, cuda):
    import torch
    L = litho_lib
    srv = L.Server(16 << 30, max_slots=4, max_queue=64)
    reqs = _request_set(3)
    tickets, outs = [], []
    for r in reqs:
        out = np.full((r["n"], r["n"]), np.nan, dtype=np.float32)
        t, loss = srv.submit(r["kind"], L.make_optics(**r["optics"]), r["n"], r["pixel"], 0.0, r["k"], r["input"],
                             out, target_host=r["target"], precision=r["precision"])
        tickets.append(t)
        outs.append((out, loss))
    status, _ = _wait_all(srv, L, tickets)
    assert all(status[t] == L.OK for t in tickets), status
    stats = srv.stats()
    assert stats["completed"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0
    assert stats["kernel_sets_cached"] >= 2
    srv.close()
    # each result equals the same request run alone through the direct C-ABI calls
    for r, (out, loss) in zip(reqs, outs):
        kern = L.litho_make_kernels(L.make_optics(**r["optics"]), r["n"], r["pixel"], [0.0], r["k"])
        x = torch.from_numpy(r["input"][None]).to(cuda)
        if r["kind"] == "image":
            ref = L.litho_aerial(kern, x, precision=r["precision"]).cpu().numpy()[0, 0]
            assert np.abs(out - ref).max() <= 1e-6
        else:
            g, lo = L.litho_ilt_grad(kern, x, torch.from_numpy(r["target"][None]).to(cuda),
                                     precision="fft32/coarse")  # the server's ILT steps
            assert np.abs(out - g.cpu().numpy()[0]).max() <= 1e-6 * max(1e-30, np.abs(out).max())
            assert abs(loss[0] - lo[0]) <= 1e-9 * lo[0]


def test_admission_rejections_cancel_and_injected_failure(litho_lib, cuda):
    L = litho_lib
    big = np.zeros((2048, 2048), dtype=np.float32)
    out = np.zeros_like(big)
    tiny = L.Server(1 << 20, max_slots=1, max_queue=4)
    with pytest.raises(L.LithoError) as e:
        L._check(_submit_raw(tiny, L, "image", DUV, 2048, 8.0, 8, big, out))
    assert e.value.status == L.EINVAL
    tiny.close()

    srv = L.Server(8 << 30, max_slots=1, max_queue=2)
    a_in = np.zeros((2048, 2048), dtype=np.float32)
    a_out = np.zeros_like(a_in)
    # kernels for these optics are not built yet, so both requests stay queued for a while
    t1, _ = srv.submit("image", L.make_optics(**DUV), 2048, 8.0, 10.0, 24, a_in, a_out)
    t2, _ = srv.submit("image", L.make_optics(**DUV), 2048, 8.0, 20.0, 24, a_in.copy(), a_out.copy())
    with pytest.raises(L.LithoError) as e:
        srv.submit("image", L.make_optics(**DUV), 2048, 8.0, 30.0, 24, a_in.copy(), a_out.copy())
    assert e.value.status == L.EBUSY
    assert srv.cancel(t2) == L.OK
    assert srv.poll(t2, 0) == L.ECANCELED
    assert srv.poll(t1, 120000) == L.OK
    # injected allocation failure: that request fails with ENOMEM, the next one runs
    srv.inject_fault(1)
    m = synth.random_rect_mask(256, seed=5)
    o1 = np.zeros_like(m)
    o2 = np.zeros_like(m)
    f1, _ = srv.submit("image", L.make_optics(**DUV), 256, 8.0, 0.0, 8, m, o1)
    assert srv.poll(f1, 60000) == L.ENOMEM
    f2, _ = srv.submit("image", L.make_optics(**DUV), 256, 8.0, 0.0, 8, m, o2)
    assert srv.poll(f2, 60000) == L.OK and np.abs(o2).max() > 0
    s = srv.stats()
    assert s["rejected"] >= 1 and s["cancelled"] == 1
    srv.close()


def _submit_raw(srv, L, kind, optics, n, pixel, k, inp, out):
    r = L.litho_request()
    r.kind = L.REQ_IMAGE if kind == "image" else L.REQ_ILT_STEP
    r.optics = L.make_optics(**optics)
    r.n, r.pixel_nm, r.defocus_nm, r.k, r.precision, r.dose = n, pixel, 0.0, k, 0, 1.0
    r.input_host = inp.ctypes.data
    r.output_host = out.ctypes.data
    t = L.c_uint64()
    return L.lib().litho_serve_submit(srv.handle, L.byref(r), L.byref(t))


def test_small_requests_overtake_large_ones(litho_lib, cuda):
    """Head-of-line independence: small images submitted after twelve large ILT steps
    (three batches of full-grid 2048^2 steps on three of the four slots) finish before
    the last of them; small batches run on high-priority streams.  Kernel sets are warmed
    first and the large requests use page-locked buffers (no staging copies on the host),
    so that only execution time counts."""
    import torch
    L = litho_lib
    srv = L.Server(16 << 30, max_slots=4, max_queue=64)
    keep = []

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
        keep.append(t)
        return t.numpy()

    big_in, big_tg = synth.ilt_clip(2048, 8.0, seed=1)
    big_in, big_tg = pinned(big_in), pinned(big_tg)
    small = synth.random_rect_mask(256, seed=2)
    warm = [srv.submit("ilt", L.make_optics(**DUV), 2048, 8.0, 0.0, 24, big_in, pinned(np.zeros_like(big_in)),
                       target_host=big_tg)[0],
            srv.submit("image", L.make_optics(**DUV), 256, 8.0, 0.0, 8, small, np.zeros_like(small))[0]]
    st, _ = _wait_all(srv, L, warm)
    assert all(v == L.OK for v in st.values())
    outs = [pinned(np.zeros_like(big_in)) for _ in range(12)]
    big = [srv.submit("ilt", L.make_optics(**DUV), 2048, 8.0, 0.0, 24, big_in, outs[i],
                      target_host=big_tg)[0] for i in range(12)]
    ts = [srv.submit("image", L.make_optics(**DUV), 256, 8.0, 0.0, 8, small, np.zeros_like(small))[0]
          for _ in range(6)]
    st, order = _wait_all(srv, L, big + ts)
    assert all(v == L.OK for v in st.values())
    assert max(order.index(t) for t in ts) < max(order.index(t) for t in big), order
    srv.close()


def test_injected_slow_request_does_not_hold_the_others(litho_lib, cuda):
    """A request made slow on its own slot (a fixed device delay) finishes
    last while the requests submitted after it complete on the other slots,
    all with the same result as the request run alone."""
    L = litho_lib
    srv = L.Server(16 << 30, max_slots=4, max_queue=64)
    opt = L.make_optics(**DUV)
    m = synth.random_rect_mask(256, seed=7)
    ref = np.zeros_like(m)
    t, _ = srv.submit("image", opt, 256, 8.0, 0.0, 8, m, ref)    # builds and warms the kernel set
    assert srv.poll(t, 60000) == L.OK
    srv.inject_fault(2)
    outs = [np.zeros_like(m) for _ in range(4)]
    tickets = [srv.submit("image", opt, 256, 8.0, 0.0, 8, m, outs[i])[0] for i in range(4)]
    status, order = _wait_all(srv, L, tickets, timeout_s=120)
    assert all(status[t] == L.OK for t in tickets), status
    assert order[-1] == tickets[0], order
    for o in outs:
        assert np.array_equal(o, ref)
    srv.close()


def test_queued_requests_of_one_key_run_as_batches(litho_lib, cuda):
    """Continuous batching: while a slow request holds the only slot, 24 images and 6 ILT
    steps of one kernel set queue up (half of the images in pinned buffers, half pageable);
    when the slot frees they run as grouped calls, far fewer than one per request, and each
    result is bit-identical to the request run alone."""
    import torch
    L = litho_lib
    srv = L.Server(16 << 30, max_slots=1, max_queue=256)
    opt = L.make_optics(**DUV)
    m0 = synth.random_rect_mask(256, seed=9)
    t, _ = srv.submit("image", opt, 256, 8.0, 0.0, 8, m0, np.zeros_like(m0))    # builds the kernel set
    assert srv.poll(t, 60000) == L.OK
    srv.inject_fault(2)                       # the next request holds the only slot for 200 ms
    hold, _ = srv.submit("image", opt, 256, 8.0, 0.0, 8, m0, np.zeros_like(m0))
    srv.stats_reset()
    keep, jobs = [], []
    for i in range(24):
        m = synth.random_rect_mask(256, seed=300 + i)
        if i % 2:
            mp = torch.from_numpy(m).pin_memory()
            op = torch.zeros_like(mp).pin_memory()
            keep += [mp, op]
            m, out = mp.numpy(), op.numpy()
        else:
            out = np.zeros_like(m)
        tk, _ = srv.submit("image", opt, 256, 8.0, 0.0, 8, m, out)
        jobs.append(("image", tk, m, None, out, None))
    for i in range(6):
        th, tg = synth.ilt_clip(256, 8.0, seed=700 + i)
        th, tg = np.ascontiguousarray(th), np.ascontiguousarray(tg)
        out = np.zeros_like(th)
        tk, loss = srv.submit("ilt", opt, 256, 8.0, 0.0, 8, th, out, target_host=tg)
        jobs.append(("ilt", tk, th, tg, out, loss))
    status, _ = _wait_all(srv, L, [hold] + [j[1] for j in jobs], timeout_s=120)
    assert all(v == L.OK for v in status.values()), status
    s = srv.stats()
    print(f"batches {s['batches']} for {s['completed']} requests, largest {s['max_batch']}")
    assert s["max_batch"] >= 6 and s["batches"] <= 8
    srv.close()
    kern = L.litho_make_kernels(opt, 256, 8.0, [0.0], 8)
    for kind, _, x, tg, out, loss in jobs:
        xd = torch.from_numpy(np.ascontiguousarray(x)[None]).to(cuda)
        if kind == "image":
            assert np.array_equal(out, L.litho_aerial(kern, xd).cpu().numpy()[0, 0])
        else:
            g, lo = L.litho_ilt_grad(kern, xd, torch.from_numpy(tg[None]).to(cuda), precision="fft32/coarse")
            assert np.array_equal(out, g.cpu().numpy()[0]) and loss[0] == lo[0]
