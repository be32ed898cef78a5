"""The continuous-batching render server (multi-user conferencing, Sec. 3 / Sec. 6).

Each request rendered in the mix must equal the same request rendered alone
through nr_set_pose + nr_render; admission respects the memory budget; every
wait is bounded; malformed requests are refused on the host.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2306_16541_gb300 import synth

from _util import nrmod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def subjects():
    return [synth.subject(900 + i, hash_scale=0.5, res_last_std=0.02, with_ellipsoids=True) for i in range(3)]


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        res = int(rng.choice([24, 40, 64]))
        cam = synth.camera(res, res, 1.25 * res, synth.random_eye(rng), int(rng.choice([16, 32])), 0.5, 4.5)
        aa, rt = synth.random_pose(rng)
        out.append(dict(subject=int(rng.integers(3)), cam=cam, aa=aa, rt=rt,
                        mlp=["f32", "bf16", "f32", "fp8"][k % 4], occ=bool(k % 3 != 0)))
    return out


@pytest.mark.parametrize("order", ["edf", "smallest_first", "fifo"])
def test_mix_equals_alone(subjects, order):
    """Under every dispatch policy each request of the mix equals the same request rendered
    alone, bit for bit (bf16 and fp8 requests on the tcgen05 pipeline included)."""
    nr = nrmod()
    subs = [nr.Subject(s) for s in subjects]
    srv = nr.Server(max_bytes=8 << 30, max_slots=6)
    try:
        srv.set_policy(order={"edf": nr.NR_SERVE_EDF, "smallest_first": nr.NR_SERVE_SMALLEST_FIRST,
                              "fifo": nr.NR_SERVE_FIFO}[order], priority_streams=(order == "smallest_first"))
        for s in subs:
            srv.add_subject(s)
        reqs = _requests(30, 1)
        outs, ids = [], []
        for q in reqs:
            out = torch.full((q["cam"].height, q["cam"].width, 4), float("nan"), device="cuda")
            opts = nr.make_opts(q["mlp"], "f32", q["occ"], 1e-4)
            ids.append(srv.submit(srv.request(q["subject"], q["cam"], q["aa"], q["rt"], opts, out)))
            outs.append(out)
        lat = [srv.wait(i, 60000) for i in ids]
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["failed"] == 0
        assert st["peak_active"] > 1                    # requests really overlapped on the device
        assert st["bytes_in_use"] >= st["slots"] * (1 << 30)   # the budget allows 2^20-ray chunks
        assert all(l > 0 for l in lat)
        for q, out in zip(reqs, outs):
            S = subs[q["subject"]]
            S.set_pose(q["aa"], q["rt"])
            alone = S.render(q["cam"], nr.make_opts(q["mlp"], "f32", q["occ"], 1e-4))
            torch.cuda.synchronize()
            assert torch.equal(out, alone)
    finally:
        srv.close()
        for s in subs:
            s.close()


def test_admission_by_memory_budget_and_pinned_host_output(subjects):
    nr = nrmod()
    S = nr.Subject(subjects[0])
    one_slot = 137 << 20                                # the budget holds exactly one slot
    srv = nr.Server(max_bytes=one_slot, max_slots=8)
    try:
        srv.add_subject(S)
        reqs = _requests(6, 2)
        outs, ids = [], []
        for q in reqs:
            out = torch.zeros(q["cam"].height, q["cam"].width, 4).pin_memory()
            ids.append(srv.submit(srv.request(0, q["cam"], q["aa"], q["rt"], nr.make_opts("f32"), out)))
            outs.append(out)
        for i in ids:
            srv.wait(i, 60000)
        st = srv.stats()
        assert st["slots"] == 1 and st["peak_active"] == 1 and st["completed"] == 6
        assert st["bytes_in_use"] <= one_slot               # 2^17-ray chunks: larger frames take several
        q = reqs[-1]
        S.set_pose(q["aa"], q["rt"])
        assert torch.equal(outs[-1], S.render(q["cam"], nr.make_opts("f32")).cpu())
    finally:
        srv.close()
        S.close()


def test_frames_larger_than_a_chunk_equal_the_plain_render(subjects):
    """A 512 x 384 request (196,608 rays) on a server whose budget allows only 2^17-ray chunks is
    rendered in two passes; the image equals nr_render's single pass bit for bit."""
    nr = nrmod()
    S = nr.Subject(subjects[2])
    srv = nr.Server(max_bytes=137 << 20, max_slots=1)
    try:
        srv.add_subject(S)
        rng = np.random.default_rng(77)
        cam = synth.camera(512, 384, 480.0, synth.random_eye(rng), 32, 0.5, 4.5)
        aa, rt = synth.random_pose(rng)
        for mlp in ("f32", "bf16"):
            opts = nr.make_opts(mlp, "f32", True, 1e-4)
            out = torch.full((384, 512, 4), float("nan"), device="cuda")
            srv.wait(srv.submit(srv.request(0, cam, aa, rt, opts, out)), 60000)
            S.set_pose(aa, rt)
            alone = S.render(cam, opts)
            torch.cuda.synchronize()
            assert torch.equal(out, alone), mlp
        assert srv.stats()["bytes_in_use"] <= 137 << 20
    finally:
        srv.close()
        S.close()


def test_bounded_waits_and_refusals(subjects):
    nr = nrmod()
    S = nr.Subject(subjects[1])
    srv = nr.Server(max_bytes=1 << 30, max_slots=1)
    try:
        srv.add_subject(S)
        cam = synth.camera(256, 256, 320.0, (0.0, 0.0, 2.5), 128, 0.5, 4.5)
        aa, rt = synth.random_pose(np.random.default_rng(3))
        outs = [torch.zeros(256, 256, 4, device="cuda") for _ in range(8)]
        ids = [srv.submit(srv.request(0, cam, aa, rt, nr.make_opts("f32"), o)) for o in outs]
        lat = C.c_double()
        rc = nr.lib.nr_server_wait(srv.h, ids[-1], 0, C.byref(lat))
        assert rc in (nr.NR_ETIMEOUT, nr.NR_OK)         # a zero-length wait never blocks
        with pytest.raises(nr.NRError) as e:            # pageable host output is refused
            srv.submit(srv.request(0, cam, aa, rt, nr.make_opts(), np.zeros((256, 256, 4), np.float32).ctypes.data))
        assert e.value.code == nr.NR_EINVAL
        with pytest.raises(nr.NRError) as e:
            srv.submit(srv.request(7, cam, aa, rt, nr.make_opts(), outs[0]))
        assert e.value.code == nr.NR_EINVAL
        bad = aa.copy()
        bad[3, 1] = np.nan
        with pytest.raises(nr.NRError):
            srv.submit(srv.request(0, cam, bad, rt, nr.make_opts(), outs[0]))
        srv.stop(120000)                                # drains the queue, then the worker exits
        for i in ids:
            assert srv.poll(i)[0] == 2
        with pytest.raises(nr.NRError) as e:
            srv.submit(srv.request(0, cam, aa, rt, nr.make_opts(), outs[0]))
        assert e.value.code == nr.NR_ESTATE
    finally:
        srv.close()
        S.close()
