"""Same-level ghost exchange (host logic).

Within one level of the hierarchy (Section 4), every ghost cell of a patch
that lies over the interior of a sibling patch -- or over a periodic image of
one -- takes the sibling's value; the remaining ghost cells are the
coarse-fine boundary (filled by prolongation, ``ctu_prolong``) or the
physical boundary.  ``plan`` lists the copies as boxes in the layout of the
library's ``ctu_copy_box``; ``split`` divides them between processes that
own disjoint sets of patches; ``exchange`` performs one exchange with the
copy, pack and unpack operations and the point-to-point transport passed in
(the library's ``ctu_copy`` / ``ctu_pack`` / ``ctu_unpack`` and
``torch.distributed`` on the GPU).

Patch coordinates: ``lo`` is the first interior cell in the level's index
space, ``n`` the interior extent, ``base`` the pool offset of the patch's
first (ghost) cell in its owner's pool.  Box coordinates are the
destination patch's interior coordinates (ghosts at -4..-1 and n..n+3); the
source cell of destination cell x is x + shift in the source patch.
"""
from __future__ import annotations

import itertools

import numpy as np

GHOST = 4


def plan(patches, domain, periodic, ndim):
    """patches: list of (lo[3], n[3], base); domain: the level's extent in
    cells (3 ints); periodic: 3 bools.  Returns a list of box dicts with
    keys dst, src (patch indices), dn, sn, lo, hi, shift, dbase, sbase,
    ordered by destination, then periodic image, then source."""
    lo = np.array([p[0] for p in patches], dtype=np.int64)
    n = np.array([p[1] for p in patches], dtype=np.int64)
    base = [int(p[2]) for p in patches]
    g = np.array([GHOST if d < ndim else 0 for d in range(3)], dtype=np.int64)
    images = [[0] + ([-int(domain[d]), int(domain[d])] if periodic[d] and d < ndim else []) for d in range(3)]
    shifts = [np.array(s, dtype=np.int64) for s in itertools.product(*images)]
    out = []
    for i in range(len(patches)):
        glo, ghi = lo[i] - g, lo[i] + n[i] + g
        for s in shifts:
            slo, shi = lo + s, lo + n + s  # source interiors, shifted
            blo = np.maximum(glo[None, :], slo)
            bhi = np.minimum(ghi[None, :], shi)
            hit = np.all(blo < bhi, axis=1)
            if not np.any(s):
                hit[i] = False  # a patch's own interior
            for j in np.nonzero(hit)[0]:
                out.append({"dst": i, "src": int(j), "dn": [int(v) for v in n[i]], "sn": [int(v) for v in n[j]],
                            "lo": [int(v) for v in blo[j] - lo[i]], "hi": [int(v) for v in bhi[j] - lo[i]],
                            "shift": [int(v) for v in lo[i] - lo[j] - s],
                            "dbase": base[i], "sbase": base[int(j)]})
    return out


def cells(box):
    return int(np.prod([h - l for l, h in zip(box["lo"], box["hi"])]))


def split(boxes, owner, rank):
    """The boxes rank `rank` copies locally, and per peer the boxes it packs
    and sends (its patches are the sources) and the boxes it receives and
    unpacks (its patches are the destinations), each in plan order, so both
    sides of a pair agree on the buffer layout."""
    local, send, recv = [], {}, {}
    for b in boxes:
        od, os_ = owner[b["dst"]], owner[b["src"]]
        if od == rank and os_ == rank:
            local.append(b)
        elif os_ == rank:
            send.setdefault(od, []).append(b)
        elif od == rank:
            recv.setdefault(os_, []).append(b)
    return local, send, recv


def exchange(boxes, owner, rank, U, copy, pack, unpack, sendrecv):
    """One exchange on rank `rank`: the local copies, then per peer (in
    increasing rank) pack -> sendrecv -> unpack.  copy(U, boxes),
    pack(U, boxes) -> buffer, unpack(U, buffer, boxes) and
    sendrecv(peer, sendbuf, nrecv) -> recvbuf are supplied by the caller."""
    local, send, recv = split(boxes, owner, rank)
    if local:
        copy(U, local)
    for peer in sorted(set(send) | set(recv)):
        sb = pack(U, send.get(peer, []))
        nr = 9 * sum(cells(b) for b in recv.get(peer, []))
        rb = sendrecv(peer, sb, nr)
        if recv.get(peer):
            unpack(U, rb, recv[peer])


def torch_sendrecv(like):
    """A sendrecv for ``exchange`` over the default torch.distributed
    process group (NCCL on the GPU, gloo on the CPU): one isend/irecv pair
    per peer.  `like` is a tensor whose dtype and device the buffers take."""
    import torch
    import torch.distributed as dist

    def sr(peer, sendbuf, nrecv):
        sb = sendbuf if torch.is_tensor(sendbuf) else torch.as_tensor(sendbuf)
        sb = sb.to(like.device, like.dtype).contiguous()
        rb = torch.empty(nrecv, dtype=like.dtype, device=like.device)
        ops = []
        if sb.numel():
            ops.append(dist.P2POp(dist.isend, sb, peer))
        if nrecv:
            ops.append(dist.P2POp(dist.irecv, rb, peer))
        for w in dist.batch_isend_irecv(ops) if ops else []:
            w.wait()
        return rb

    return sr


def _subtract(r, c):
    """Box r minus box c as disjoint boxes ((lo, hi) lists of 3 ints)."""
    lo, hi = list(r[0]), list(r[1])
    if any(max(lo[d], c[0][d]) >= min(hi[d], c[1][d]) for d in range(3)):
        return [r]
    out = []
    for d in range(3):
        if lo[d] < c[0][d]:
            a, b = list(lo), list(hi)
            b[d] = c[0][d]
            out.append((a, b))
            lo[d] = c[0][d]
        if hi[d] > c[1][d]:
            a, b = list(lo), list(hi)
            a[d] = c[1][d]
            out.append((a, b))
            hi[d] = c[1][d]
    return out


def ghost_slabs(n, ndim):
    """The ghost shell of a patch as 2 ndim disjoint boxes (patch
    coordinates): along d, the two slabs of 4 layers, spanning the interior
    in the dimensions before d and the ghosted extent in those after it."""
    g = [GHOST if d < ndim else 0 for d in range(3)]
    out = []
    for d in range(ndim):
        for lo_d, hi_d in ((-GHOST, 0), (n[d], n[d] + GHOST)):
            lo = [lo_d if e == d else (0 if e < d else -g[e]) for e in range(3)]
            hi = [hi_d if e == d else (n[e] if e < d else n[e] + g[e]) for e in range(3)]
            out.append((lo, hi))
    return out


def uncovered(boxes, npatch, sizes, ndim):
    """Per patch, the ghost cells no exchange box writes, as disjoint boxes
    (patch coordinates): the coarse-fine and physical boundary, left to
    prolongation and boundary conditions.  sizes[i] is patch i's n."""
    cover = [[] for _ in range(npatch)]
    for b in boxes:
        cover[b["dst"]].append((b["lo"], b["hi"]))
    out = []
    for i in range(npatch):
        rest = ghost_slabs(sizes[i], ndim)
        for c in cover[i]:
            rest = [p for r in rest for p in _subtract(r, c)]
        out.append(rest)
    return out


def ship_registers(items, rank, reg, sendrecv):
    """Flux-register windows to the rank that applies the reflux (Eq.
    fluxcorr, addreflux): a fine window accumulates on the rank that owns
    the fine patch, while the correction lands on the coarse patch's owner.
    items: (src_rank, src_off, dst_rank, dst_off, size) per window whose two
    ranks differ (doubles of the register arrays); every rank passes the same
    list.  reg: this rank's register array (a 1-D tensor); the received
    windows overwrite reg[dst_off : dst_off + size] (ranges a rank receives
    must not overlap ranges it sends).  Per peer, in increasing rank, one
    sendrecv of the windows in list order."""
    import torch
    send, recv = {}, {}
    for it in items:
        s, so, d, do, n = it
        if s == rank and d != rank:
            send.setdefault(d, []).append((so, n))
        elif d == rank and s != rank:
            recv.setdefault(s, []).append((do, n))
    for peer in sorted(set(send) | set(recv)):
        parts = [reg[o:o + n] for o, n in send.get(peer, [])]
        sb = torch.cat(parts) if parts else reg[:0]
        nr = sum(n for _, n in recv.get(peer, []))
        rb = sendrecv(peer, sb, nr)
        pos = 0
        for o, n in recv.get(peer, []):
            reg[o:o + n] = rb[pos:pos + n]
            pos += n
