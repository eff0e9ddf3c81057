"""Helpers of the GPU parity tests: run the CUDA path through the C ABI with
its intermediates dumped, and replay each stage in the CPU oracle from the
GPU's own inputs to that stage."""
from __future__ import annotations

import numpy as np

from oracle import rabitq as R

U64_MAX = np.uint64(0xFFFFFFFFFFFFFFFF)


def lib():
    import paper_2605_16007_gb300 as rq

    rq.build()
    return rq


def host_index(ix) -> dict:
    """The GPU index as an oracle index dict (arrays copied to the host)."""
    h = ix.to_host()
    return dict(n=h["n"], dim=h["dim"], dp=h["dp"], nlist=h["nlist"], P=h["P"],
                centroids=h["centroids"], cR=h["cR"], offsets=h["offsets"],
                ids=h["ids"], assign=h["assign"], codes=h["codes"], r=h["r"],
                alpha=h["alpha"], r2=h["factors"][:, 0].copy(),
                f=h["factors"][:, 1].copy(), raw=h["raw"].astype(np.float32))


def search_dump(ix, q, nprobe, k, n_rerank, mixed=False, **kw):
    """rq_search (or rq_search_mixed) with every intermediate dumped."""
    import torch

    nq = q.shape[0]
    npb = np.broadcast_to(np.asarray(nprobe, np.int32), (nq,))
    kk = np.broadcast_to(np.asarray(k, np.int32), (nq,))
    nr = np.broadcast_to(np.asarray(n_rerank, np.int32), (nq,))
    npmax = int(npb.max())
    nsel = np.where(nr > 0, nr, kk)
    nsmax = int(nsel.max())
    kmax = int(kk.max())
    hv = ix.view()
    dp, cb = hv["dim_pad"], hv["code_bytes"]
    dev = torch.device("cuda")
    d = dict(
        qrot=torch.empty((nq, dp), dtype=torch.float32, device=dev),
        probe_ids=torch.empty((nq, npmax), dtype=torch.int32, device=dev),
        probe_dist=torch.empty((nq, npmax), dtype=torch.float32, device=dev),
        qparams=torch.empty((nq, npmax, 4), dtype=torch.float32, device=dev),
        planes=torch.empty((nq, npmax, 4, cb), dtype=torch.uint8, device=dev),
        bound=torch.empty((nq,), dtype=torch.int32, device=dev),
        selected=torch.empty((nq, nsmax), dtype=torch.int64, device=dev),
        n_candidates=torch.empty((nq,), dtype=torch.int32, device=dev),
    )
    qd = torch.from_numpy(np.ascontiguousarray(q, np.float32)).to(dev)
    ids = torch.empty((nq, kmax), dtype=torch.int64, device=dev)
    dist = torch.empty((nq, kmax), dtype=torch.float32, device=dev)
    if mixed or not (np.all(npb == npb[0]) and np.all(kk == kk[0]) and np.all(nr == nr[0])):
        ix.search_mixed(qd, npb, kk, nr, k_stride=kmax, out_ids=ids, out_dist=dist,
                        dump=d, **kw)
    else:
        ix.search(qd, int(npb[0]), int(kk[0]), int(nr[0]), out_ids=ids, out_dist=dist,
                  dump=d, **kw)
    torch.cuda.synchronize()
    out = {name: t.cpu().numpy() for name, t in d.items()}
    out["bound"] = out["bound"].view(np.uint32)
    out["selected"] = out["selected"].view(np.uint64)
    out["ids"] = ids.cpu().numpy()
    out["dist"] = dist.cpu().numpy()
    out["npb"], out["kk"], out["nr"], out["nsel"] = npb, kk, nr, nsel
    return out


def replay_and_compare(hix: dict, q: np.ndarray, dump: dict, prune: bool = True,
                       check_probe: bool = True, estimator: str = "bq4"):
    """Recompute every stage in the oracle from the GPU's inputs to it and
    require bit-equality. Returns counts of compared items. With
    estimator="lut" the per-pair quantities are nq2 and the residual sum
    (no planes)."""
    nq = q.shape[0]
    npmax = dump["probe_ids"].shape[1]
    stats = dict(pairs=0, candidates=0)
    if check_probe:
        pid, pd = R.probe(dump["qrot"], hix["cR"], npmax)
        assert np.array_equal(pid, dump["probe_ids"]), "probe ids differ"
        assert np.array_equal(pd.view(np.uint32), dump["probe_dist"].view(np.uint32)), \
            "probe distances differ"
    for i in range(nq):
        np_i = int(dump["npb"][i])
        pids = dump["probe_ids"][i, :np_i].astype(np.int64)
        d2, cid, qs = R.list_candidates(hix, dump["qrot"][i], pids, estimator)
        for p, qz in enumerate(qs):
            gp = dump["qparams"][i, p]
            if estimator == "lut":
                res = np.asarray(qz, np.float32)
                assert gp[2:3].view(np.uint32)[0] == R.lane_sum(res * res).view(np.uint32), (i, p, "nq2")
                assert gp[3:4].view(np.uint32)[0] == R.lane_sum(res).view(np.uint32), (i, p, "sum")
                stats["pairs"] += 1
                continue
            assert gp[0] == qz["vl"][0] and gp[1] == qz["delta"][0], (i, p, "vl/delta")
            assert gp[2].view(np.uint32) == qz["nq2"][0].view(np.uint32), (i, p, "nq2")
            assert gp[3:4].view(np.int32)[0] == qz["sq"][0], (i, p, "Sq")
            assert np.array_equal(dump["planes"][i, p], qz["planes"][0]), (i, p, "planes")
            stats["pairs"] += 1
        n_sel = int(dump["nsel"][i])
        tau = R.first_bound(d2, n_sel) if prune else R.U32_MAX
        assert int(dump["bound"][i]) == int(tau), (i, "bound")
        npass = int(np.count_nonzero(R.orderable(d2) <= np.uint64(tau)))
        assert int(dump["n_candidates"][i]) == npass, (i, "candidates passing the bound")
        sel = R.select_candidates(d2, cid, n_sel, prune)
        stats.setdefault("estimates", []).append(d2)
        gsel = np.sort(dump["selected"][i, :n_sel])   # a set when re-ranked
        assert np.array_equal(gsel[:sel.size], sel), (i, "selected keys")
        assert np.all(gsel[sel.size:] == U64_MAX), (i, "selection padding")
        stats["candidates"] += d2.size
        k = int(dump["kk"][i])
        if dump["nr"][i] > 0:
            oi, od = R.rerank(hix["raw"], q[i], R.key_id(sel), k)
        else:
            oi = np.full(k, -1, np.int64)
            od = np.full(k, np.inf, np.float32)
            oi[:min(k, sel.size)] = R.key_id(sel[:k])
            od[:min(k, sel.size)] = R.key_dist(sel[:k])
        assert np.array_equal(dump["ids"][i, :k], oi), (i, "final ids")
        assert np.array_equal(dump["dist"][i, :k].view(np.uint32), od.view(np.uint32)), \
            (i, "final distances")
        if dump["ids"].shape[1] > k:
            assert np.all(dump["ids"][i, k:] == -1) and np.all(np.isinf(dump["dist"][i, k:]))
    return stats
