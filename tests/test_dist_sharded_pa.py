"""Within-run sharding of one population across ranks (the multi-GPU design
for a run larger than one GPU), exercised with two and three gloo ranks on
CPU around the oracle's per-replica pieces. Rank r holds a contiguous slice
of the replica slots. Every step it

  1. all-reduces the integer energy histogram (exact, order-free) and
     computes the same S, F, U tables as every other rank (Eq. Q,
     Eq. resampling-factors);
  2. draws the copy numbers of its own old slots from the RESAMPLE words of
     their global slot indices;
  3. all-gathers the shard totals, giving the global offset of its copies
     (copies keep old-slot order, so the concatenation is the one-process
     population);
  4. sends each copy to the rank whose equal contiguous slice holds its new
     slot (point-to-point);
  5. sweeps its slice with SWEEP words keyed by the global new-slot index and
     all-reduces the integer moment sums for the row.

The rows (bit for bit) and the final population equal the single-process
oracle's: sharding changes where replicas live, not any result."""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

CFG = dict(L=8, R=600, theta=3, beta_f=0.6, dbeta=0.1, seed=23)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _sum_ints(vals):
    t = torch.tensor(list(vals), dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [int(v) for v in t.tolist()]


def _families(fam):
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, fam.tolist())
    return int(np.unique(np.concatenate([np.asarray(f, dtype=np.int64) for f in out])).size)


def _migrate(pop, fam, first, R_new):
    """Copies hold global new slots [first, first + n); return this rank's
    equal slice [R_new r / G, R_new (r+1) / G) after point-to-point sends."""
    G, r = dist.get_world_size(), dist.get_rank()
    n = pop.shape[0]
    slices = [(R_new * q // G, R_new * (q + 1) // G) for q in range(G)]
    starts = [0] * G
    dist.all_gather_object(starts, (first, n))
    lo, hi = slices[r]
    L = pop.shape[1]
    out_pop = np.empty((hi - lo, L, L), dtype=np.int8)
    out_fam = np.empty(hi - lo, dtype=np.int64)
    reqs, keep = [], []
    for q in range(G):  # my copies that belong to rank q
        a, b = max(first, slices[q][0]), min(first + n, slices[q][1])
        if a >= b:
            continue
        seg_pop, seg_fam = pop[a - first:b - first], fam[a - first:b - first]
        if q == r:
            out_pop[a - lo:b - lo], out_fam[a - lo:b - lo] = seg_pop, seg_fam
        else:
            tp, tf = torch.from_numpy(np.ascontiguousarray(seg_pop)), torch.from_numpy(np.ascontiguousarray(seg_fam))
            keep += [tp, tf]
            reqs += [dist.isend(tp, q), dist.isend(tf, q)]
    for q in range(G):  # rank q's copies that belong to me
        qf, qn = starts[q]
        a, b = max(qf, lo), min(qf + qn, hi)
        if q == r or a >= b:
            continue
        tp = torch.empty((b - a, L, L), dtype=torch.int8)
        tf = torch.empty(b - a, dtype=torch.int64)
        dist.recv(tp, q)
        dist.recv(tf, q)
        out_pop[a - lo:b - lo], out_fam[a - lo:b - lo] = tp.numpy(), tf.numpy()
    for q in reqs:
        q.wait()
    return out_pop, out_fam, lo


def _sharded_run(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle.pa_oracle import (copy_tables, init_spins, level_weights, make_row, measure, metropolis_threshold,
                                  moment_sums, normaliser_S, resample_words, sweep)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L, R, theta, seed = CFG["L"], CFG["R"], CFG["theta"], CFG["seed"]
    N = L * L
    n_steps = int(round(CFG["beta_f"] / CFG["dbeta"]))
    lo = R * rank // world
    slots = np.arange(lo, R * (rank + 1) // world, dtype=np.int64)
    pop = init_spins(L, slots, seed)
    E, M = measure(pop)
    fam = slots.copy()
    rows, sum_lnQ, R_prev = [], 0.0, R
    rows.append(make_row(0.0, N, R, _sum_ints(moment_sums(E, M)), 0.0, 0.0, _families(fam)))
    for i in range(1, n_steps + 1):
        beta, delta = i * CFG["dbeta"], CFG["dbeta"]
        lv = (E + 2 * N) // 4
        H = np.array(_sum_ints(np.bincount(lv, minlength=N + 1).tolist()), dtype=np.int64)
        occ = np.nonzero(H)[0]
        kmin, kmax = int(occ[0]), int(occ[-1])
        t = level_weights(delta, kmax - kmin + 1)
        S = normaliser_S(H, kmin, kmax, t, N)
        _, F, U = copy_tables(R, t, S)
        x = resample_words(seed, i, R_prev).astype(np.int64)[lo:lo + E.size]  # words of my global old slots
        d = lv - kmin
        r = F[d] + (x < U[d]).astype(np.int64)
        totals = [0] * world
        dist.all_gather_object(totals, int(r.sum()))
        first, R_new = sum(totals[:rank]), sum(totals)
        idx = np.repeat(np.arange(E.size), r)
        pop, fam, lo = _migrate(pop[idx], fam[idx], first, R_new)
        pop = np.ascontiguousarray(pop)
        sweep(pop, np.arange(lo, lo + pop.shape[0], dtype=np.int64), seed, (i - 1) * theta, theta,
              metropolis_threshold(beta, 4), metropolis_threshold(beta, 8))
        E, M = measure(pop)
        lnQ = (math.log(S) - math.log(float(R_prev))) - delta * float(-2 * N + 4 * kmin)
        sum_lnQ += lnQ
        rows.append(make_row(beta, N, R_new, _sum_ints(moment_sums(E, M)), sum_lnQ, lnQ, _families(fam)))
        R_prev = R_new
    parts = [None] * world
    dist.all_gather_object(parts, pop)
    if rank == 0:
        queue.put(([rw.as_tuple() for rw in rows], np.concatenate(parts)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_population_equals_one_process(world):
    from oracle.pa_oracle import PopulationAnnealing
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_run, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    rows, pop = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref = PopulationAnnealing(CFG["L"], CFG["R"], CFG["theta"], beta_f=CFG["beta_f"], dbeta=CFG["dbeta"],
                              seed=CFG["seed"])
    ref.run()
    assert rows == [r.as_tuple() for r in ref.rows]
    np.testing.assert_array_equal(pop, ref.pop)
