"""Host logic of the multi-process path on CPU: point shards cover the run
exactly once, and the gloo all-gather combination of per-rank sums (and of
per-rank histograms) gives every rank the same bits, equal to one process
over all points up to the rounding of the combination."""
import math
import os
import socket

import numpy as np
import pytest

from paper_0908_4403_gb300 import dist as D
from paper_0908_4403_gb300 import heget as H

SEED = 0x0908440300008000


def test_shards_cover_every_point_once():
    for N in (0, 1, 7, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            seen = []
            for rank in range(world):
                i0, n = D.shard(N, world, rank)
                seen.extend(range(i0, i0 + n))
            assert seen == list(range(N))
    with pytest.raises(ValueError):
        D.shard(10, 2, 2)


def _result_from_weights(w, tries, kind):
    """A heget_xsec_result built directly from per-event weights (math.fsum)."""
    r = H.heget_xsec_result()
    r.sum_w, r.sum_w2 = math.fsum(w), math.fsum(x * x for x in w)
    r.n_pass = int(np.count_nonzero(w))
    r.n_total, r.n_tries = len(w), int(np.sum(tries))
    return D.combine([r], kind)


def _shard_weights(oracle, n, N, world, rank):
    i0, cnt = D.shard(N, world, rank)
    w, _, tries = oracle.event_weights(n, SEED, i0, cnt, oracle.toy_pdf(), oracle.cuts(), threads=1)
    return w, tries


def test_combine_of_shards_equals_one_run(oracle):
    n, N = 3, 3001
    w, _, tries = oracle.event_weights(n, SEED, 0, N, oracle.toy_pdf(), oracle.cuts(), threads=2)
    whole = _result_from_weights(w, tries, H.HEGET_SAMPLER_TOY_PDF)
    for world in (2, 3, 5):
        parts = []
        for rank in range(world):
            i0, cnt = D.shard(N, world, rank)
            parts.append(_result_from_weights(w[i0:i0 + cnt], tries[i0:i0 + cnt], H.HEGET_SAMPLER_TOY_PDF))
        got = D.combine(parts, H.HEGET_SAMPLER_TOY_PDF)
        assert got.n_total == N and got.n_tries == whole.n_tries and got.n_pass == whole.n_pass
        assert got.sum_w == pytest.approx(whole.sum_w, rel=4e-16, abs=0)
        assert got.sigma_fb == pytest.approx(whole.sigma_fb, rel=1e-15, abs=0)
        assert got.err_fb == pytest.approx(whole.err_fb, rel=1e-12, abs=0)
    # toy-PDF scale: 2 x acceptance
    assert whole.sigma_fb == pytest.approx(2 * (N / whole.n_tries) * whole.sum_w / N, rel=1e-15)


def _rank_main(rank, world, port, n, N, out_dir):
    import torch.distributed as dist
    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, tries = _shard_weights(O, n, N, world, rank)
        mine = _result_from_weights(w, tries, H.HEGET_SAMPLER_TOY_PDF)
        tot = D.allreduce_result(mine, H.HEGET_SAMPLER_TOY_PDF)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([tot.sigma_fb, tot.err_fb, tot.sum_w, tot.sum_w2, tot.n_total, tot.n_tries, tot.n_pass]))
        i0, cnt = D.shard(N, world, rank)
        ps = O.phase_space(n, SEED, i0, cnt, O.toy_pdf(), O.cuts())
        flat = np.concatenate([h.ravel() for h in O.hist(n, ps["momenta"], ps["y"], w, HSPECS)])
        np.save(os.path.join(out_dir, f"h{rank}.npy"), D.allreduce_hist(flat))
    finally:
        dist.destroy_process_group()


HSPECS = [(0, 20, 20.0, 420.0), (3, 16, 0.0, 8.0)]


def _shard_hist(oracle, n, N, world, rank):
    i0, cnt = D.shard(N, world, rank)
    w, _ = _shard_weights(oracle, n, N, world, rank)
    ps = oracle.phase_space(n, SEED, i0, cnt, oracle.toy_pdf(), oracle.cuts())
    return np.concatenate([h.ravel() for h in oracle.hist(n, ps["momenta"], ps["y"], w, HSPECS)])


def test_combined_shard_histograms_equal_one_run(oracle):
    n, N = 3, 1501
    whole = _shard_hist(oracle, n, N, 1, 0)
    for world in (2, 3):
        got = D.combine_hists([_shard_hist(oracle, n, N, world, r) for r in range(world)])
        np.testing.assert_allclose(got, whole, rtol=1e-15, atol=0)
    with pytest.raises(ValueError):
        D.combine_hists([np.zeros(4), np.zeros(6)])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2])
def test_gloo_allreduce_gives_every_rank_the_single_process_result(oracle, tmp_path, world):
    import torch.multiprocessing as mp
    n, N = 3, 2001
    mp.spawn(_rank_main, args=(world, _free_port(), n, N, str(tmp_path)), nprocs=world, join=True)
    got = [np.load(tmp_path / f"r{r}.npy") for r in range(world)]
    for g in got[1:]:
        assert np.array_equal(g.view(np.uint64), got[0].view(np.uint64))   # same bits on every rank
    parts = [_result_from_weights(*_shard_weights(oracle, n, N, world, r), H.HEGET_SAMPLER_TOY_PDF)
             for r in range(world)]
    ref = D.combine(parts, H.HEGET_SAMPLER_TOY_PDF)
    assert got[0][0] == ref.sigma_fb and got[0][2] == ref.sum_w and int(got[0][4]) == N
    hs = [np.load(tmp_path / f"h{r}.npy") for r in range(world)]
    for h in hs[1:]:
        assert np.array_equal(h.view(np.uint64), hs[0].view(np.uint64))   # same bits on every rank
    ref_h = D.combine_hists([_shard_hist(oracle, n, N, world, r) for r in range(world)])
    assert np.array_equal(hs[0], ref_h)


def test_combine_refusals():
    """The library refuses an unknown sampler kind and histograms of different
    layouts; an empty combination is the empty result."""
    with pytest.raises(H.HegetError):
        H.heget_xsec_combine([H.heget_xsec_result()], 7)
    empty = D.combine([], H.HEGET_SAMPLER_FIXED)
    assert empty.n_total == 0 and empty.sigma_fb == 0.0 and empty.err_fb == 0.0
    with pytest.raises(ValueError):
        D.combine_hists([np.zeros(3), np.zeros(4)])
