"""Frequency-sharded application of Eq. FFT_v2 over several ranks (one GPU each).

The hybrid method's steps split along two different axes:

* the row transforms (x) of Eq. FFT_v2 work plane by plane, a plane being one
  (state, layer, component) of m;
* the column transforms (y), the sum over the source layers and the inverse
  column transforms work kx column by kx column, every plane at once, with the
  tensor of that kx.

So each rank transforms the rows of its own contiguous range of planes, one
all-to-all turns plane-major row spectra into kx-slab-major ones, each rank runs
the column steps on its own slab of kx (holding only that slab of the tensor:
the tensor, the largest array of a many-layer stack, is divided among the
ranks), a second all-to-all returns the slabs, and each rank runs the inverse
row transforms of its planes.  The exchanges land in local memory (no remote
loads, no multicast): 2 x the row spectrum per apply in total.

This module holds the partitioning and the two exchanges.  The three local
steps are passed in as callables (on a GPU: `gpu_steps`, the library's row and
slab kernels through demag_rows_forward, demag_columns_slab and
demag_rows_inverse; the CPU tests pass stand-ins), so the orchestration runs
unchanged over NCCL or gloo process groups.
"""


def even_ranges(n, parts):
    """Split range(n) into `parts` contiguous ranges whose sizes differ by at most
    one (the first n mod parts ranges one longer).  Returns [(start, stop)]."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    q, r = divmod(n, parts)
    out, s = [], 0
    for k in range(parts):
        e = s + q + (1 if k < r else 0)
        out.append((s, e))
        s = e
    return out


class ShardedApply:
    """One rank's part of a sharded apply.

    P planes (B * L * 3 of a batch), Kx stored x-frequencies, ny rows of a
    plane's row spectrum.  The callables:

      rows_forward(p0, p1) -> complex tensor [p1 - p0, Kx, ny]: the row
          spectrum of planes p0..p1-1 (this rank's planes);
      columns_slab(slab)   : complex tensor [P, k1 - k0, ny] of every plane at
          this rank's x-frequencies k0..k1-1, transformed in place (column
          transforms, layer sum, inverse column transforms);
      rows_inverse(spec, p0, p1): the field of planes p0..p1-1 from their row
          spectrum [p1 - p0, Kx, ny].

    dist is a torch.distributed module with an initialised process group (or
    None for one rank).
    """

    def __init__(self, P, Kx, ny, rank, world, rows_forward, columns_slab, rows_inverse, dist=None,
                 stage_host=False):
        self.P, self.Kx, self.ny = P, Kx, ny
        self.rank, self.world = rank, world
        self.planes = even_ranges(P, world)
        self.slabs = even_ranges(Kx, world)
        self.rows_forward, self.columns_slab, self.rows_inverse = rows_forward, columns_slab, rows_inverse
        self.dist = dist
        self.stage_host = stage_host  # exchange through host memory (gloo ranks with device spectra)

    def bytes_exchanged(self, itemsize):
        """Bytes this rank sends per apply (both exchanges), complex items of `itemsize`."""
        p0, p1 = self.planes[self.rank]
        k0, k1 = self.slabs[self.rank]
        own = (p1 - p0) * self.Kx * self.ny - (p1 - p0) * (k1 - k0) * self.ny
        back = self.P * (k1 - k0) * self.ny - (p1 - p0) * (k1 - k0) * self.ny
        return (own + back) * itemsize

    def _exchange(self, send_blocks, recv_shapes, like):
        """all-to-all of complex blocks (send_blocks[d] to rank d, recv block s
        of shape recv_shapes[s]); the blocks travel as real pairs."""
        import torch
        if self.world == 1:
            return [send_blocks[0]]
        send = torch.cat([torch.view_as_real(b.contiguous()).reshape(-1) for b in send_blocks])
        home = send.device
        if self.stage_host:
            send = send.cpu()
        in_sizes = [2 * b.numel() for b in send_blocks]
        out_sizes = [2 * int(torch.Size(s).numel()) for s in recv_shapes]
        recv = torch.empty(sum(out_sizes), dtype=send.dtype, device=send.device)
        self.dist.all_to_all_single(recv, send, out_sizes, in_sizes)
        recv = recv.to(home)
        out, o = [], 0
        for s, n in zip(recv_shapes, out_sizes):
            out.append(torch.view_as_complex(recv[o:o + n].view(*s, 2)))
            o += n
        return out

    def apply(self):
        """Run the three local steps and the two exchanges; returns this rank's
        row spectrum after the column steps (its planes, every kx)."""
        import torch
        p0, p1 = self.planes[self.rank]
        k0, k1 = self.slabs[self.rank]
        spec = self.rows_forward(p0, p1)                      # [np, Kx, ny]
        # plane-major -> slab-major: to rank d go my planes at d's frequencies
        blocks = self._exchange([spec[:, a:b, :] for a, b in self.slabs],
                                [(q1 - q0, k1 - k0, self.ny) for q0, q1 in self.planes], spec)
        slab = torch.cat(blocks, dim=0) if len(blocks) > 1 else blocks[0].contiguous()  # [P, nk, ny]
        self.columns_slab(slab)
        # slab-major -> plane-major: to rank d go d's planes at my frequencies
        back = self._exchange([slab[a:b] for a, b in self.planes],
                              [(p1 - p0, b - a, self.ny) for a, b in self.slabs], slab)
        for (a, b), blk in zip(self.slabs, back):
            spec[:, a:b, :] = blk
        self.rows_inverse(spec, p0, p1)
        return spec


def gpu_steps(plan, m, H, B, Ms, k0, k1, stream=None):
    """The three local steps of a ShardedApply on the library's kernels.

    plan: a ._lib.Plan on the split path whose tensor covers x-frequencies
    k0..k1-1 (this rank's slab; after Plan.keep_slab(k0, k1) it holds nothing
    else); m, H: the batch's device fields [B, L, 3, ny, nx] (this rank reads
    and writes only its planes of them).  Returns (rows_forward, columns_slab,
    rows_inverse) for ShardedApply."""
    import torch
    from . import _lib
    info = plan.info
    Kx, ny = info["Px"] // 2 + 1, info["ny"]
    cdt = torch.complex128 if info["precision"] == _lib.PREC_FP64 else torch.complex64

    def rows_forward(p0, p1):
        spec = torch.empty(p1 - p0, Kx, ny, dtype=cdt, device=m.device)
        return _lib.demag_rows_forward(plan.handle, m, p0, p1, spec, stream, info)

    def columns_slab(slab):
        _lib.demag_columns_slab(plan.handle, slab, k0, k1, B, stream, info)

    def rows_inverse(spec, p0, p1):
        _lib.demag_rows_inverse(plan.handle, spec, p0, p1, Ms, H, stream, info)

    return rows_forward, columns_slab, rows_inverse
