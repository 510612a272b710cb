"""The partition of one lattice into slabs of whole domain planes along z,
one per rank (the decomposition of Sec. 3.1 that a multi-GPU run of a single
lattice would use), checked on CPU with 2 gloo ranks against the oracle run
in one process.  No GPU needed.

Each rank holds its slab's spins and one halo plane of sites above and below.
Per cycle (Sec. 3.1 steps 1-6, eight colours in rotation, Sec. 3.2 step 4a):
every active domain of the slab forms its frequency line from the spins
(step 1); the ranks take the maximum of their largest R_k with one
allreduce-max of one double (step 2); every active domain draws its event on
the line padded to R_max (steps 3-4) and flips its site; every rank advances
the same clock (step 5); then the boundary planes go to the neighbouring
ranks as their halos (step 6).  Gathered, the slabs must equal the oracle's
lattice bit for bit, with the same clock and counters."""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def slab_run(rank, world, L, d, J, H, T, seed, ncycles):
    import oracle
    nd = L // d
    planes = nd // world                          # domain planes of this rank
    z0, z1 = rank * planes * d, (rank + 1) * planes * d  # its site planes
    full = oracle.init_spins(L, seed).reshape(L, L, L)   # [z][y][x], site x + L (y + L z)
    s = full[z0:z1].astype(np.int8).copy()
    halo_lo, halo_hi = full[(z0 - 1) % L].copy(), full[z1 % L].copy()
    r = oracle.rates(J, H, T)
    clock, nflip, nnull = 0.0, 0, 0
    for t in range(ncycles):
        # step 1: classes of the slab's sites (up neighbours, the halo planes at the slab faces)
        up = (np.concatenate([halo_lo[None], s, halo_hi[None]]) > 0).astype(np.int64)
        mid = up[1:-1]
        u = (np.roll(mid, 1, 2) + np.roll(mid, -1, 2) + np.roll(mid, 1, 1) + np.roll(mid, -1, 1)
             + up[:-2] + up[2:])
        cls = 7 * (s > 0).astype(np.int64) + u
        col = t % 8
        lines = []
        for dz in range(z0 // d, z1 // d):
            for dy in range(nd):
                for dx in range(nd):
                    if ((dx & 1) | (dy & 1) << 1 | (dz & 1) << 2) != col:
                        continue
                    k = dx + nd * (dy + nd * dz)
                    sites = []
                    for l in range(d ** 3):
                        x, y, z = l % d, (l // d) % d, l // (d * d)
                        sites.append((dz * d + z - z0, dy * d + y, dx * d + x))
                    c_of = [int(cls[p]) for p in sites]
                    n = [0] * 14
                    for c in c_of:
                        n[c] += 1
                    cum, acc = [], 0.0
                    for c in range(14):
                        acc = acc + n[c] * float(r[c])
                        cum.append(acc)
                    lines.append((k, sites, c_of, n, cum))
        # step 2: R_max over the active domains of every slab, one double
        rm = torch.tensor([max(cum[13] for *_, cum in lines)], dtype=torch.float64)
        dist.all_reduce(rm, op=dist.ReduceOp.MAX)
        R = float(rm.item())
        # steps 3-4 and 6: the events, all from the pre-flip state, then the flips
        flips = []
        for k, sites, c_of, n, cum in lines:
            w = [int(x) for x in oracle.philox((t, k, 1, 0), (seed, 0))]
            target = (w[0] >> 11) * 2.0 ** -53 * R
            chosen = next((c for c in range(14) if target < cum[c]), -1)
            if chosen < 0:
                nnull += 1
                continue
            j = (w[1] * n[chosen]) >> 64
            flips.append([p for p, c in zip(sites, c_of) if c == chosen][j])
            nflip += 1
        for p in flips:
            s[p] = -s[p]
        # step 5: the same clock on every rank
        wc = int(oracle.philox((t, 0, 2, 0), (seed, 0))[0])
        clock = clock + (-math.log((2 * (wc >> 12) + 1) * 2.0 ** -53) / R)
        # step 6: the boundary planes become the neighbours' halos
        faces = torch.from_numpy(np.stack([s[0], s[-1]]).astype(np.int8))
        got = [torch.empty_like(faces) for _ in range(world)]
        dist.all_gather(got, faces)
        halo_lo = got[(rank - 1) % world][1].numpy().copy()  # top plane of the rank below
        halo_hi = got[(rank + 1) % world][0].numpy().copy()  # bottom plane of the rank above
    slabs = [torch.empty(planes * d * L * L, dtype=torch.int8) for _ in range(world)]
    dist.all_gather(slabs, torch.from_numpy(s.reshape(-1).copy()))
    cnt = torch.tensor([nflip, nnull], dtype=torch.int64)
    dist.all_reduce(cnt)
    return np.concatenate([x.numpy() for x in slabs]), clock, int(cnt[0]), int(cnt[1])


def _worker(rank, world, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spins, clock, nf, nn = slab_run(rank, world, *case)
        out.put((rank, spins.tobytes(), clock, nf, nn))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", [
    (8, 2, 1.0, 0.0, 4.5115, 31, 17),     # 2 domain planes per rank
    (16, 2, 1.0, 0.05, 3.8, 32, 12),      # 4 per rank, H != 0
    (16, 4, -0.8, 0.0, 2.6, 33, 9),       # 2 per rank, antiferromagnetic
])
def test_two_slabs_equal_the_single_lattice(case):
    import oracle
    L, d, J, H, T, seed, n = case
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    st = oracle.State(L, d, J, H, T, seed)
    st.run(n)
    for rank, spins, clock, nf, nn in res:
        assert np.array_equal(np.frombuffer(spins, dtype=np.int8), st.spins), rank
        assert clock == st.clock, (rank, clock, st.clock)
        assert (nf, nn) == (st.n_flip, st.n_null)
