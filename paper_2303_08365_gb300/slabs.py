"""Slab decomposition of one grid along its slowest axis, with one halo
exchange per block of Tb steps.

The paper's concurrent scheduler splits one grid between workers and keeps
the communication small in two ways (Sec. 5.3): only the halo regions cross
between workers, and the halo of a whole block of Tb time steps is sent in
one centralised message instead of Tb small ones (k messages of n_b bytes
cost k(alpha + n_b beta), one message of k n_b bytes alpha + k n_b beta).
Here the workers are slabs of the slowest axis (z in 3D, y in 2D, the only
axis in 1D), one per GPU (or several on one device), and the exchange moves
r*Tb planes each way per block:

  - slab k owns planes [z0_k, z1_k) and keeps a local array of its owned
    planes plus H = r*Tb halo planes on each side that has a neighbour (no
    halo at the outer faces of a Dirichlet grid, whose zero ghost cells the
    local sweep supplies itself; a periodic grid's first and last slabs are
    neighbours);
  - per block: every halo is refreshed from the neighbour's owned edge
    planes (device-local copies in one process, point-to-point send/receive
    between ranks), then each slab advances its local array by the block's
    steps (Tb, or the remainder) with the library's own sweep on that array;
  - after s steps the outer r*s planes of each halo hold values computed from
    the array's own edge (wrong there), but the owned planes depend only on
    planes within r*s <= H of them, which were all correct at the start of
    the block: the owned planes are exactly the single-grid result.  The
    kernels apply the same per-cell multiply-add chain whatever the array's
    shape, so they are bitwise equal to it too;
  - the halo is recomputed by both neighbours (2H planes per slab and step):
    the price of one message per block instead of one per step.

Everything here is host-side scheduling; every time step runs in the CUDA
kernels behind Plan.run, and the halo planes are moved by cudaMemcpyAsync
(torch copies) or NCCL (torch.distributed).  The local step is a parameter so
that the same schedule can be exercised on CPU with a reference step.
"""
import numpy as np


def slab_bounds(n, nslabs):
    """Near-equal split of n planes into nslabs contiguous ranges [z0, z1)."""
    if nslabs < 1 or nslabs > n:
        raise ValueError(f"cannot cut {n} planes into {nslabs} slabs")
    base, extra = divmod(n, nslabs)
    out, z = [], 0
    for k in range(nslabs):
        m = base + (1 if k < extra else 0)
        out.append((z, z + m))
        z += m
    return out


class SlabLayout:
    """Where every plane of every slab's local array comes from.

    shape: the global grid shape (slowest axis first); radius, Tb: halo depth
    H = radius * Tb; periodic: the boundary rule.
    """

    def __init__(self, shape, nslabs, radius, Tb, periodic):
        self.shape = tuple(int(s) for s in shape)
        self.n = self.shape[0]
        self.nslabs = int(nslabs)
        self.radius = int(radius)
        self.Tb = int(Tb)
        self.periodic = bool(periodic)
        self.H = self.radius * self.Tb
        self.bounds = slab_bounds(self.n, self.nslabs)
        self.halo = []  # (below, above) halo planes of each slab's local array
        for k, (z0, z1) in enumerate(self.bounds):
            if self.nslabs == 1:
                lo = hi = 0  # the whole grid: the local sweep applies the boundary rule itself
            else:
                lo = self.H if (self.periodic or k > 0) else 0
                hi = self.H if (self.periodic or k < self.nslabs - 1) else 0
            if (lo or hi) and z1 - z0 < self.H:
                raise ValueError(f"slab {k} owns {z1 - z0} planes, fewer than the halo depth {self.H}")
            self.halo.append((lo, hi))

    def owned(self, k):
        return self.bounds[k][1] - self.bounds[k][0]

    def local_shape(self, k):
        lo, hi = self.halo[k]
        return (lo + self.owned(k) + hi,) + self.shape[1:]

    def owned_slice(self, k):
        """Planes of slab k's local array that it owns."""
        lo = self.halo[k][0]
        return slice(lo, lo + self.owned(k))

    def messages(self):
        """One exchange: (src slab, src local planes, dst slab, dst local
        planes) for every halo, each a slice of the slowest axis."""
        msgs = []
        for k in range(self.nslabs):
            lo, hi = self.halo[k]
            n_k = self.owned(k)
            if lo:
                s = (k - 1) % self.nslabs
                ls, ns = self.halo[s][0], self.owned(s)
                msgs.append((s, slice(ls + ns - self.H, ls + ns), k, slice(0, self.H)))
            if hi:
                s = (k + 1) % self.nslabs
                ls = self.halo[s][0]
                msgs.append((s, slice(ls, ls + self.H), k, slice(lo + n_k, lo + n_k + self.H)))
        return msgs

    def block_steps(self, T):
        """Steps of each block: Tb until the remainder."""
        out, t = [], 0
        while t < T:
            s = min(self.Tb, T - t)
            out.append(s)
            t += s
        return out


class LocalSlabs:
    """All slabs of one grid in one process (one device, or one per device):
    the exchange is a device-to-device copy per halo.

    arrays: the slabs' local arrays (torch tensors or numpy arrays) of
    layout.local_shape(k); step(k, array, steps) advances slab k's array in
    place.  `make_gpu_steps` builds the default step from the library's plans.
    """

    def __init__(self, layout, arrays, step):
        self.layout = layout
        self.arrays = list(arrays)
        self.step = step
        self.exchanges = 0

    @classmethod
    def scatter(cls, layout, grid, step, devices=None):
        """Local arrays filled with the owned planes of `grid` (torch, any
        device; the halos are filled by the first exchange)."""
        import torch
        arrays = []
        for k, (z0, z1) in enumerate(layout.bounds):
            dev = grid.device if devices is None else torch.device(devices[k])
            a = torch.zeros(layout.local_shape(k), dtype=grid.dtype, device=dev)
            a[layout.owned_slice(k)].copy_(grid[z0:z1])
            arrays.append(a)
        return cls(layout, arrays, step)

    def exchange(self):
        for s, ss, d, ds in self.layout.messages():
            src = self.arrays[s][ss]
            dst = self.arrays[d][ds]
            if hasattr(dst, "copy_"):
                dst.copy_(src, non_blocking=True)  # cudaMemcpyAsync (peer copy across devices)
            else:
                dst[...] = src
        self.exchanges += 1

    def run(self, T):
        for steps in self.layout.block_steps(T):
            self.exchange()
            for k, a in enumerate(self.arrays):
                self.step(k, a, steps)

    def gather(self, out):
        for k, (z0, z1) in enumerate(self.layout.bounds):
            src = self.arrays[k][self.layout.owned_slice(k)]
            if hasattr(out, "copy_"):
                out[z0:z1].copy_(src)
            else:
                out[z0:z1] = src
        return out


def make_gpu_steps(layout, radius, weights, boundary, tuning=None):
    """Step functions backed by one library plan per slab (local shape, same
    stencil and boundary rule, optional (Tb, variant) tuning); returns
    (step, plans)."""
    import paper_2303_08365_gb300 as st
    plans = [st.Plan(layout.local_shape(k), radius, weights, boundary) for k in range(layout.nslabs)]
    if tuning is not None:
        for p in plans:
            p.set_tuning(*tuning)

    def step(k, array, steps):
        plans[k].run(array, steps)

    return step, plans


class DistSlab:
    """This rank's slab of a grid decomposed over a torch.distributed group:
    rank k owns slab k.  The exchange posts every send and receive of the
    block's halos at once (isend/irecv of contiguous plane blocks: NCCL for
    CUDA tensors, gloo for host tensors) and waits for them."""

    def __init__(self, layout, array, step, group=None):
        import torch.distributed as dist
        self.layout = layout
        self.array = array
        self.step = step
        self.group = group
        self.rank = dist.get_rank(group)
        if dist.get_world_size(group) != layout.nslabs:
            raise ValueError("one slab per rank")
        self.exchanges = 0

    def exchange(self):
        import torch.distributed as dist
        reqs = []
        for s, ss, d, ds in self.layout.messages():
            if s == d == self.rank:  # a periodic slab that is its own neighbour
                self.array[ds].copy_(self.array[ss])
            elif s == self.rank:
                reqs.append(dist.isend(self.array[ss].contiguous(), dst=d, group=self.group))
            elif d == self.rank:
                buf = self.array[ds]
                if not buf.is_contiguous():
                    raise ValueError("halo planes must be contiguous")
                reqs.append(dist.irecv(buf, src=s, group=self.group))
        for r in reqs:
            r.wait()
        self.exchanges += 1

    def run(self, T):
        for steps in self.layout.block_steps(T):
            self.exchange()
            self.step(self.rank, self.array, steps)

    def owned(self):
        return self.array[self.layout.owned_slice(self.rank)]


def message_bytes(layout, itemsize=8):
    """Bytes one exchange moves (every halo once)."""
    plane = int(np.prod(layout.shape[1:])) * itemsize
    return sum((ss.stop - ss.start) * plane for _, ss, _, _ in layout.messages())
