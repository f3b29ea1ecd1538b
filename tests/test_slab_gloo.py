"""The z-slab split of one simulation (§4.4) run as separate CPU ranks over gloo.

The library's partition (heat_slab_plan, host-only) gives each rank one slab;
each rank keeps its owned node layers plus one ghost layer per neighbour,
exactly as the GPU slab form lays out its buffers (include/heat.h). Per CG
iteration the ranks exchange one node layer of u = P^-1 r and x with their
neighbours (send/recv) and merge both inner products of the
Chronopoulos-Gear iteration into ONE all_reduce; the true residual is
recomputed every 50 iterations and on convergence, and a step closes on it.
The local operator on each rank is the oracle's element-by-element product
on the slab's own sub-mesh. The fields gathered from the owned layers must
equal the unsplit oracle solution (sparse LU) within the FP64 parity bar, and
every iteration must have cost exactly one all_reduce.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import workloads as W
    return W.random_box(6, 5, 9, seed=23, dirichlet={4: 1.0, 0: -0.5}, flux={5: 1.0, 2: 0.4}, theta=0.5,
                        dt=0.01, nsteps=3, flux_steps=2, rtol=1e-12, contrast=(0.2, 5.0))


def _local(p, r, S, first):
    """The slab's sub-problem: element layers [kg0, top), ghost layers included."""
    import workloads as W
    lo, hi = r > 0, r < S - 1
    kg0 = first[r] - (1 if lo else 0)
    top = first[r + 1] if hi else p.nz
    nzl = top - kg0
    hz = p.extent[2] / p.nz
    plane = p.nx * p.ny
    keep = lambda f: f < 4 or (f == 4 and not lo) or (f == 5 and not hi)  # noqa: E731
    q = W.Problem(f"slab{r}", p.nx, p.ny, nzl, origin=(p.origin[0], p.origin[1], p.origin[2] + kg0 * hz),
                  extent=(p.extent[0], p.extent[1], nzl * hz), rho_c=p.rho_c[plane * kg0: plane * top],
                  k=p.k[plane * kg0: plane * top],
                  dirichlet={f: v for f, v in p.dirichlet.items() if keep(f)},
                  flux={f: v for f, v in p.flux.items() if keep(f)}, flux_steps=p.flux_steps,
                  theta=p.theta, dt=p.dt, rtol=p.rtol)
    own0 = 1 if lo else 0
    own1 = nzl - 1 if hi else nzl
    return q, kg0, own0, own1


class Counter:
    n = 0


def _allreduce(vals):
    t = torch.tensor(vals, dtype=torch.float64)
    dist.all_reduce(t)
    Counter.n += 1
    return t.tolist()


def _exchange(vec, r, S, own0, own1, pxy, nzl):
    """Owned boundary layers to the neighbours' ghost layers."""
    reqs, bufs = [], []
    if r > 0:
        reqs.append(dist.isend(torch.from_numpy(vec[own0 * pxy:(own0 + 1) * pxy].copy()), r - 1))
        bufs.append((0, torch.empty(pxy, dtype=torch.float64)))
        reqs.append(dist.irecv(bufs[-1][1], r - 1))
    if r < S - 1:
        reqs.append(dist.isend(torch.from_numpy(vec[own1 * pxy:(own1 + 1) * pxy].copy()), r + 1))
        bufs.append((nzl, torch.empty(pxy, dtype=torch.float64)))
        reqs.append(dist.irecv(bufs[-1][1], r + 1))
    for q in reqs:
        q.wait()
    for layer, b in bufs:
        vec[layer * pxy:(layer + 1) * pxy] = b.numpy()


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_1905_07622_gb300.api as api
        from oracle import fem, transient
        p = _problem()
        first = api.heat_slab_plan(p.nz, world)
        q, kg0, own0, own1 = _local(p, rank, world, first)
        pxy = (p.nx + 1) * (p.ny + 1)
        nzl = q.nz
        nl = q.n_nodes
        owned = np.zeros(nl, dtype=bool)
        owned[own0 * pxy:(own1 + 1) * pxy] = True
        dir_ids, dir_vals = fem.dirichlet_nodes(q)
        free = np.ones(nl, dtype=bool)
        free[dir_ids] = False
        rows = owned & free
        idt, th = 1.0 / p.dt, p.theta
        A_all = lambda x: fem.apply_all(q, x, idt, th, eliminate=False)  # noqa: E731
        pinv = 1.0 / fem.diagonal_all(q, idt, th)
        F = fem.flux_vector(q)
        g = np.zeros(nl)
        g[dir_ids] = dir_vals
        lift = A_all(g)
        u0 = np.array(p.u0)
        gd, gv = fem.dirichlet_nodes(p)
        u0[gd] = gv
        u1 = u0[pxy * kg0: pxy * (kg0 + nzl + 1)].copy()
        u2 = None
        steps = []
        for n in range(1, p.nsteps + 1):
            b = fem.apply_all(q, u1, idt, th - 1.0, eliminate=False) - lift
            if transient.flux_on(p, n):
                b = b + F
            b[~free] = 0.0
            (delta_b,) = _allreduce([float(np.sum((b * b * pinv)[rows]))])
            thresh = p.rtol ** 2 * delta_b
            x = u1.copy() if u2 is None else 2.0 * u1 - u2

            def true_residual():  # b carries the lift: Dirichlet columns are dropped here
                r = np.where(free, b - fem.apply_all(q, x, idt, th, eliminate=True), 0.0)
                u = pinv * r
                _exchange(u, rank, world, own0, own1, pxy, nzl)
                (gam,) = _allreduce([float(np.sum((r * u)[rows]))])
                return r, u, gam

            r, u, gam = true_residual()
            it, since, restart = 0, 0, True
            calls0 = Counter.n
            pv = np.zeros(nl)
            sv = np.zeros(nl)
            gam_old = alpha_old = 0.0
            extra = 0  # all_reduces of true-residual passes
            detect = 0  # merged reductions that found the recurrence converged
            while gam > thresh:
                w = fem.apply_all(q, u, idt, th, eliminate=True)
                w[~free] = 0.0
                gam, dlt = _allreduce([float(np.sum((r * u)[rows])), float(np.sum((w * u)[rows]))])
                if gam <= thresh:
                    detect += 1
                    r, u, gam = true_residual()
                    extra += 1
                    since = 0
                    continue
                if restart:
                    beta, alpha = 0.0, gam / dlt
                else:
                    beta = gam / gam_old
                    alpha = gam / (dlt - beta * gam / alpha_old)
                gam_old, alpha_old, restart = gam, alpha, False
                pv = u + beta * pv
                sv = w + beta * sv
                x = x + alpha * pv
                r = r - alpha * sv
                u = pinv * r
                _exchange(u, rank, world, own0, own1, pxy, nzl)
                _exchange(x, rank, world, own0, own1, pxy, nzl)
                it += 1
                since += 1
                if since >= 50:
                    r, u, gam = true_residual()
                    extra += 1
                    since = 0
            per_iter_calls = Counter.n - calls0 - extra - detect
            _exchange(x, rank, world, own0, own1, pxy, nzl)
            steps.append((x[own0 * pxy:(own1 + 1) * pxy].copy(), it, per_iter_calls))
            u2, u1 = u1, x
        out.put((rank, kg0 + own0, kg0 + own1, steps))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_ranks_match_unsplit_oracle_with_one_allreduce_per_iteration(world):
    from oracle import transient
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    p = _problem()
    ref = transient.run(p, solver="direct")
    pxy = (p.nx + 1) * (p.ny + 1)
    covered = np.zeros(p.n_nodes, dtype=int)
    fields = [np.zeros(p.n_nodes) for _ in range(p.nsteps)]
    iters = {}
    for rank, l0, l1, steps in got:
        covered[l0 * pxy:(l1 + 1) * pxy] += 1
        for n, (vals, it, calls) in enumerate(steps):
            fields[n][l0 * pxy:(l1 + 1) * pxy] = vals
            iters.setdefault(n, set()).add(it)
            assert calls == it, (rank, n, calls, it)  # one all_reduce per iteration
    assert np.all(covered == 1)  # the owned layers partition the mesh
    for n in range(p.nsteps):
        assert len(iters[n]) == 1  # every rank ran the same iterations
        err = np.linalg.norm(fields[n] - ref.u[n + 1]) / np.linalg.norm(ref.u[n + 1])
        assert err <= 1e-9, (world, n, err)
