"""Protocol of the z-slab decomposition (Sec. 2.5: slabs along x3, the stage inputs' planes next to each
cut exchanged before every stage, one error maximum over all slabs for the step control) on the CPU with
two gloo ranks.  Each rank holds one slab of a full-model bead problem plus a ghost plane at the cut,
evaluates the oracle's right-hand side on its slab (the ghost plane supplies the neighbour values; its own
output is discarded), forms the Merson stage combinations on its planes, exchanges the cut planes with
send/recv and takes the error maximum with an all-reduce.  The ranks must reproduce the single-domain
oracle run bit for bit: the same accepted and rejected attempts and the same state at every cell.  The
GPU's in-process slab mode runs the same exchange schedule with copy kernels."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE = (13, 11, 16)
CUT = 7          # rank 0: planes [0, 7), rank 1: planes [7, 16)
T_END, TOL = 1.5, 1e-6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2401_01672_gb300 import inputs as I
    h = 3e-4
    sv, _ = I.packing_boolean(SHAPE, 0.5, I.uniform_radius(3.0, 5.0), 17)
    p = I.default_params(xi=h, xi_G=0.4 * h, alpha=I.ALPHA_MACRO["large"], zeta=2.0, dirichlet_faces=I.FACE_ZP,
                         theta_freeze=-5.0, theta_thaw=2.0, t_freeze=0.7)
    th0 = np.full(int(np.prod(SHAPE)), 1.0)
    ph0 = I.top_slab_indicator(SHAPE, 3)
    return h, sv * h, p, th0, ph0


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    try:
        n1, n2, n3 = SHAPE
        plane = n1 * n2
        h, sp, p, th0, ph0 = _problem()
        full = oracle.Oracle(SHAPE, h, "full", "sigmap1p", p)
        G_full = full.glass(sp, p["xi_G"])
        # this rank's planes plus one ghost plane at the cut
        k0, k1 = (0, CUT) if rank == 0 else (CUT, n3)
        e0, e1 = (k0, k1 + 1) if rank == 0 else (k0 - 1, k1)
        own = slice((k0 - e0) * plane, (k1 - e0) * plane)
        ext = oracle.Oracle((n1, n2, e1 - e0), h, "full", "sigmap1p", p)
        G = G_full[e0 * plane:e1 * plane].copy()
        mine_lo, mine_hi = own.start, own.stop
        # the plane sent to the neighbour and the ghost plane received from it
        send_sl = slice(mine_hi - plane, mine_hi) if rank == 0 else slice(mine_lo, mine_lo + plane)
        ghost_sl = slice(mine_hi, mine_hi + plane) if rank == 0 else slice(mine_lo - plane, mine_lo)
        peer = 1 - rank
        halo_bytes = 0

        def exchange(*fields):
            nonlocal halo_bytes
            for f in fields:
                buf = torch.from_numpy(f[send_sl].copy())
                got = torch.empty(plane, dtype=torch.float64)
                req = dist.isend(buf, peer)
                dist.recv(got, peer)
                req.wait()
                f[ghost_sl] = got.numpy()
                halo_bytes += 8 * plane

        th = th0[e0 * plane:e1 * plane].copy()
        ph = ph0[e0 * plane:e1 * plane].copy()
        exchange(th, ph)
        t, dt = 0.0, 0.01
        n_acc = n_rej = 0

        def rhs(ut, up):
            kt, kp = ext.rhs(G, ut, up, t)
            return kt[own], kp[own]

        while t < T_END:
            target = T_END
            if t < p["t_freeze"] and p["t_freeze"] < target:
                target = p["t_freeze"]
            step, land = dt, False
            if t + step >= target:
                step, land = target - t, True
            yt, yp = th[own], ph[own]
            k1t, k1p = rhs(th, ph)
            ut, up = th.copy(), ph.copy()
            ut[own] = yt + step / 3.0 * k1t
            up[own] = yp + step / 3.0 * k1p
            exchange(ut, up)
            k2t, k2p = rhs(ut, up)
            ut[own] = yt + step / 6.0 * k1t + step / 6.0 * k2t
            up[own] = yp + step / 6.0 * k1p + step / 6.0 * k2p
            exchange(ut, up)
            k3t, k3p = rhs(ut, up)
            ut[own] = yt + step / 8.0 * k1t + 3.0 * step / 8.0 * k3t
            up[own] = yp + step / 8.0 * k1p + 3.0 * step / 8.0 * k3p
            exchange(ut, up)
            k4t, k4p = rhs(ut, up)
            ut[own] = yt + step / 2.0 * k1t - 3.0 * step / 2.0 * k3t + 2.0 * step * k4t
            up[own] = yp + step / 2.0 * k1p - 3.0 * step / 2.0 * k3p + 2.0 * step * k4p
            exchange(ut, up)
            k5t, k5p = rhs(ut, up)
            ot = yt + step / 6.0 * (k1t + 4.0 * k4t + k5t)
            op = yp + step / 6.0 * (k1p + 4.0 * k4p + k5p)
            e = max(np.max(np.abs(step / 30.0 * (2.0 * k1t - 9.0 * k3t + 8.0 * k4t - k5t))),
                    np.max(np.abs(step / 30.0 * (2.0 * k1p - 9.0 * k3p + 8.0 * k4p - k5p))))
            E = torch.tensor([e], dtype=torch.float64)
            dist.all_reduce(E, op=dist.ReduceOp.MAX)     # one error maximum over all slabs
            E = float(E[0])
            if E <= TOL:
                t = target if land else t + step
                th[own], ph[own] = ot, op
                exchange(th, ph)
                n_acc += 1
            else:
                n_rej += 1
            dt = full.controller(E, TOL, step)
        out.put((rank, k0, k1, th[own].copy(), ph[own].copy(), t, n_acc, n_rej, halo_bytes))
    finally:
        dist.destroy_process_group()


def test_two_gloo_slabs_reproduce_the_single_domain_oracle():
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted([q.get(timeout=600) for _ in range(world)], key=lambda r: r[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    h, sp, p, th0, ph0 = _problem()
    o = oracle.Oracle(SHAPE, h, "full", "sigmap1p", p)
    G = o.glass(sp, p["xi_G"])
    ref = o.run(G, th0, ph0, 0.0, 0.01, T_END, TOL, 100000)
    assert ref["status"] == 0 and ref["t"] == T_END and ref["n_rejected"] + ref["n_accepted"] > 20
    plane = SHAPE[0] * SHAPE[1]
    for rank, k0, k1, th, ph, t, n_acc, n_rej, hb in res:
        assert (n_acc, n_rej) == (ref["n_accepted"], ref["n_rejected"])
        assert t == ref["t"]
        assert np.array_equal(th, ref["theta"][k0 * plane:k1 * plane])
        assert np.array_equal(ph, ref["phi"][k0 * plane:k1 * plane])
        # per attempt four stage exchanges of two fields, per accepted step one more, plus the first
        assert hb == 8 * plane * 2 * (1 + 4 * (n_acc + n_rej) + n_acc)
