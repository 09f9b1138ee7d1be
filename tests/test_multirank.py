"""The benchmark's multi-rank host logic on CPU with torch.distributed (gloo,
world size 2): disjoint clip shards per rank and the whole-job rate taken
over the slowest rank (the path shards by clip with no data exchange, so the
only collective is the timing reduction)."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = bench.clip_seeds(rank, 8)
    my_time = 1.0 + rank          # rank 1 is the slow one
    t = torch.tensor([my_time])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    rate = bench.whole_job_rate(8.0, world, [float(t.item())])
    q.put((rank, gathered, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, rate in out:
        a, b = gathered
        assert not set(a) & set(b) and len(a) == len(b) == 8
        assert rate == pytest.approx(16.0 / 2.0)   # 2 x 8 units over the slower rank's 2 s


def test_stage_models_are_consistent():
    peaks = {"hbm_gbs": 6785.5, "bf16_tflops_sustained": 1709.2}
    m = bench.stage_models("fp16x3/coarse", 64, 2048, 448, 3, 24, 1024, peaks)
    # split operands: Gauss's three real products (6 N'^2 C flops) per kernel and plane, each as
    # three 16-bit products; plain 16-bit operands: four real products (8 N'^2 C)
    assert m["stage2_gemm"][0] == pytest.approx(64 * 3 * 24 * 6.0 * 1024 ** 2 * 448 * 3)
    mp = bench.stage_models("fp16/coarse", 64, 2048, 448, 3, 24, 1024, peaks)
    assert mp["stage2_gemm"][0] == pytest.approx(64 * 3 * 24 * 8.0 * 1024 ** 2 * 448)
    # operands: hi and lo of Re and Im plus the hi/lo sums, 2 bytes each, per complex value
    assert m["stage2_gemm"][1] == pytest.approx(64 * 72 * 1024 * 448 * 12.0 + 64 * 3 * 1024 ** 2 * 4.0)
    # resist: 9 bytes per pixel and plane (f32 in, f32 blur and u8 printed out)
    assert m["resist"][1] == pytest.approx(64 * 3 * 2048 ** 2 * 9.0)
    assert "upsample" in m and "upsample_resist" in m
    m2 = bench.stage_models("fft32", 64, 2048, 448, 3, 24, 1024, peaks)
    assert "upsample" not in m2
    # FP32 stage 1 on the coarse grid: 8 clips per launch, so Phi is read 8 times per 64 clips
    m3 = bench.stage_models("fft32/coarse", 64, 2048, 448, 3, 24, 1024, peaks)
    assert bench.fft_group(64, 3, 24, 1024, 448) == 8
    phi, t1 = 72 * 448 ** 2 * 8.0, 64 * 72 * 1024 * 448 * 8.0
    assert m3["stage1_fft"][1] == pytest.approx(8 * phi + 64 * 448 ** 2 * 8.0 + t1)
    # on the 1024-point grid stage 2 writes each row's 2C = 896 band spectrum instead of the image
    assert m3["stage2_fft"][1] == pytest.approx(t1 + 64 * 3 * 1024 * 896 * 8.0)
    assert m3["upsample_resist"][1] == pytest.approx(64 * 3 * (1024 * 896 * 8.0 + 2048 ** 2 * 9.0))
    # roofline: the binding resource is the one with the longer time at peak
    r = bench.rooflines({"stage1_fft": (10.0, 8), "stage2_fft": (10.0, 8)}, 1, m3, peaks)
    assert r["stage1_fft"]["bound"] == "hbm" and r["stage2_fft"]["bound"] == "alu"
    assert r["stage1_fft"]["achieved"] == pytest.approx(m3["stage1_fft"][1] / 1e-2 / 1e9)


def test_ilt_models_count_the_adjoint_transforms():
    """The ILT work model: per (clip, plane, kernel) the adjoint rows take two
    transforms per row and the columns one per crop column, so the coarse grid
    (512 for 1024^2) cuts the per-kernel work about fourfold; bytes count theta,
    target and the kernels in, the gradient out."""
    import math
    fft = lambda m: 5.0 * m * math.log2(m)  # noqa: E731
    full = bench.ilt_models(16, 1024, 1024, 224, 5, 16, False, 8)
    coarse = bench.ilt_models(16, 1024, 512, 224, 5, 16, True, 8)
    per_kernel_bwd = 1024 * (2 * fft(1024) + 8.0 * 1024) + 224 * fft(1024) + 6.0 * 224 ** 2
    per_plane_bwd = 16 * per_kernel_bwd + 1024 ** 2 * 4.0 * 11
    assert full["ilt_backward"][0] == pytest.approx(16 * (224 * fft(1024) + 1024 * fft(1024) + 5 * per_plane_bwd))
    assert full["ilt_backward"][1] == pytest.approx(16 * 1024 ** 2 * 4.0)
    assert full["ilt_forward"][1] == pytest.approx(16 * 1024 ** 2 * 8.0 + 2 * 5 * 16 * 224 ** 2 * 8.0)
    ratio = full["ilt_backward"][0] / coarse["ilt_backward"][0]
    assert 2.5 < ratio < 4.5


def test_ai_models_count_both_channels():
    """The AI-input work model: the image channel (stage 1 and 2 per kernel on the evaluation
    grid) and the adjoint of ones in closed form (lam_k |Phi_k|^2 per kernel and band point, then
    the band-to-full gradient: one transform per crop column and per row, on any grid); the print
    images move 14 bytes per pixel (target and blur f32, the image read, two prints)."""
    import math
    fft = lambda m: 5.0 * m * math.log2(m)  # noqa: E731
    m = bench.ai_models(16, 2048, 1024, 448, 24, True, 21)
    mf = bench.ai_models(16, 2048, 2048, 448, 24, False, 21)
    bwd = 16 * (24 * 4.0 * 448 ** 2 + 4.0 * 448 ** 2 + 448 * fft(2048) + 2048 * fft(2048))
    assert mf["ilt_backward"][0] == pytest.approx(bwd)
    assert m["ilt_backward"][0] == pytest.approx(bwd)
    assert m["ilt_forward"][0] < mf["ilt_forward"][0] / 2
    assert m["resist"][1] == pytest.approx(16 * 2048 ** 2 * 14.0)
    assert m["ilt_forward"][1] == pytest.approx(16 * 2048 ** 2 * 12.0)
