"""Sharding the step across ranks (CPU, gloo, world size 2): each rank
traces a disjoint window of packet ids of every source (sharding.
packet_windows), the int64 deposits are summed with an all-reduce, every rank
writes the sum back and runs the per-cell update of the step, and the
result equals one rank tracing every packet, bit for bit: deposits, budget
and the four state fields.  This is the exchange a multi-device step makes
before the per-cell chemistry (packets are independent given the frozen
absorbers; integer sums do not depend on the order or the split); the CUDA
library takes the same calls (crash_write_deposits, crash_chemistry)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    import oracle
    from paper_1101_4127_gb300 import inputs
    rng = np.random.default_rng(17)
    n = 12
    E, f = inputs.blackbody_bins(1e5)
    box = inputs.Box(n=n, box_cm=6.6 * inputs.KPC_CM * n / 128,
                     nH=inputs.lognormal_field(n, 1.0, 1e-3, 17), nH0=1e-3, he_over_h=0.08,
                     x_HII0=0.2, x_HeII0=0.1, x_HeIII0=0.0, T0=5e3, isothermal=0, caseB=1,
                     z_compton=-1.0, seed=0xABCDEF, src_pos=rng.uniform(0, n, (3, 3)),
                     src_ndot=np.array([1e48, 3e47, 2e48]), bin_eV=E, bin_frac=np.tile(f, (3, 1)))
    return oracle, inputs, box, 3 * 600, 0.02 * inputs.MYR_S


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1101_4127_gb300 import sharding
    oracle, inputs, box, P, dt = _case()
    lo, hi = sharding.packet_windows(P // box.n_src, world)[rank]
    g = oracle.OracleGrid.from_box(box)
    g.set_options(chemistry=0, pkt_begin=lo, pkt_end=hi)
    g.step(dt, P)
    dep = torch.from_numpy(g.read_deposits())
    bud = torch.from_numpy(g.read(oracle.F_BUDGET)[:5].copy())
    dist.all_reduce(dep, op=dist.ReduceOp.SUM)
    dist.all_reduce(bud, op=dist.ReduceOp.SUM)
    # every rank: the summed deposits, then the step's per-cell update
    g.write_deposits(dep.numpy())
    g.chemistry(dt)
    state = np.stack([g.read(f).reshape(-1) for f in (oracle.F_XHII, oracle.F_XHEII,
                                                      oracle.F_XHEIII, oracle.F_T)])
    np.save(out + f".state{rank}.npy", state)
    if rank == 0:
        np.save(out + ".dep.npy", dep.numpy())
        np.save(out + ".bud.npy", bud.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_all_reduced_deposits_equal_single_run(tmp_path):
    out = str(tmp_path / "shard")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    oracle, inputs, box, P, dt = _case()
    g = oracle.OracleGrid.from_box(box)
    g.step(dt, P)
    assert np.array_equal(np.load(out + ".dep.npy"), g.read_deposits())
    assert np.array_equal(np.load(out + ".bud.npy"), g.read(oracle.F_BUDGET)[:5])
    state = np.stack([g.read(f).reshape(-1) for f in (oracle.F_XHII, oracle.F_XHEII,
                                                      oracle.F_XHEIII, oracle.F_T)])
    for r in range(2):
        assert np.array_equal(np.load(out + f".state{r}.npy"), state), r
