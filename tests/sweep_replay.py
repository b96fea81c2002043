"""CPU replay of an exact-order sweep schedule as the kernels receive it
(samg_sweep_schedule): bands run in an adversarial order -- always the
latest band whose next level's recorded requirements are met -- so a missing
cross-band requirement shows up as a stale read.  Inside a band the replay
follows the image: first touches read the staged copy (gathered when the
band starts) or global memory, later touches a window slot, last touches
write global memory.  It checks the image's own invariants on the way (rows
of one level write disjoint columns, a slot is read only for the column last
stored in it, a staged value is the entry's column).  Test infrastructure:
plain numpy, independent of the library's code."""
import numpy as np


def _al16(v):
    return (v + 15) & ~15


def parse(blob):
    b = memoryview(blob)
    rows, cols, nbands, nlevels, nchunks, max_slots, mode, shifted = np.frombuffer(b[:32], "<i4")
    nreq, imgb = (int(v) for v in np.frombuffer(b[32:48], "<i8"))
    at = 48
    band_chunk = np.frombuffer(b[at:at + 4 * (nbands + 1)], "<i4")
    at += 4 * (nbands + 1)
    chunks = []
    for _ in range(nchunks):
        L0, nl, nr, ne, nx, nq, nbytes, _pad = (int(v) for v in np.frombuffer(b[at:at + 32], "<i4"))
        off = int(np.frombuffer(b[at + 32:at + 40], "<i8")[0])
        chunks.append(dict(L0=L0, nl=nl, nr=nr, ne=ne, nx=nx, nq=nq, bytes=nbytes, off=off))
        at += 40
    lvl = np.frombuffer(b[at:at + 16 * nlevels], "<i4").reshape(nlevels, 4)
    at += 16 * nlevels
    req = np.frombuffer(b[at:at + 8 * nreq], "<i4").reshape(nreq, 2)
    at += 8 * nreq
    img = b[at:at + imgb]
    at += imgb
    order = np.frombuffer(b[at:at + 4 * nbands], "<i4")
    assert at + 4 * nbands == len(blob)
    return dict(rows=int(rows), cols=int(cols), nbands=int(nbands), max_slots=int(max_slots),
                mode=int(mode), shifted=bool(shifted), band_chunk=band_chunk, chunks=chunks,
                lvl=lvl, req=req, img=img, order=order)


def check_claim_order(S, ctas):
    """The tickets' band order: a permutation in which every band's required
    bands come earlier, and a claim-by-ticket run on `ctas` CTAs (a band
    holds its CTA from its claim to its last level) that finishes: at every
    step some claimed band can run its next level."""
    nb = S["nbands"]
    order = [int(v) for v in S["order"]]
    assert sorted(order) == list(range(nb)), "order is not a permutation of the bands"
    pos = {b: t for t, b in enumerate(order)}
    bc, lvl, req = S["band_chunk"], S["lvl"], S["req"]
    need = []
    for b in range(nb):
        if bc[b] == bc[b + 1]:
            need.append([])
            continue
        L0 = S["chunks"][bc[b]]["L0"]
        last = S["chunks"][bc[b + 1] - 1]
        per = []
        for L in range(L0, last["L0"] + last["nl"]):
            rq = req[lvl[L, 0]:lvl[L, 0] + lvl[L, 1]]
            for bb, _ in rq:
                assert pos[int(bb)] < pos[b], "a band's required band has a later ticket"
            per.append(rq)
        need.append(per)
    done = [0] * nb
    nxt_ticket = 0
    running = []
    while nxt_ticket < nb or running:
        while len(running) < ctas and nxt_ticket < nb:
            running.append(order[nxt_ticket])
            nxt_ticket += 1
        moved = False
        for b in list(running):
            while done[b] < len(need[b]) and all(done[int(bb)] >= int(k) for bb, k in need[b][done[b]]):
                done[b] += 1
                moved = True
            if done[b] == len(need[b]):
                running.remove(b)
                moved = True
        assert moved, "claim-by-ticket run stalls"


def _image(S, c):
    ck = S["chunks"][c]
    nl, nr, ne, nx, nq = ck["nl"], ck["nr"], ck["ne"], ck["nx"], ck["nq"]
    lq = _al16(16 * nl)
    ri = _al16(lq + 8 * nl)
    inv = _al16(ri + 8 * nr)
    ent = _al16(inv + 8 * nr)
    a = _al16(ent + 8 * ne)
    bo = _al16(a + 8 * ne)
    xc = _al16(bo + (8 * ne if S["shifted"] else 0))
    rq = _al16(xc + 4 * nx)
    total = _al16(rq + 8 * nq)
    assert total == ck["bytes"]
    m = S["img"][ck["off"]:ck["off"] + total]
    return dict(
        lv=np.frombuffer(m[:16 * nl], "<i4").reshape(nl, 4),
        lq=np.frombuffer(m[lq:lq + 8 * nl], "<i4").reshape(nl, 2),
        rq=np.frombuffer(m[rq:rq + 8 * nq], "<i4").reshape(nq, 2),
        ri=np.frombuffer(m[ri:ri + 8 * nr], "<i4").reshape(nr, 2),
        inv=np.frombuffer(m[inv:inv + 8 * nr], "<f8"),
        ent=np.frombuffer(m[ent:ent + 8 * ne], "<i4").reshape(ne, 2),
        a=np.frombuffer(m[a:a + 8 * ne], "<f8"),
        b=np.frombuffer(m[bo:bo + 8 * ne], "<f8") if S["shifted"] else np.zeros(ne),
        xc=np.frombuffer(m[xc:xc + 4 * nx], "<i4"))


def replay(S, x, rhs=None, shift=None):
    """Run the schedule on x (cols x ld, float64, updated in place)."""
    ld = x.shape[1]
    sh = np.zeros(ld) if shift is None else np.asarray(shift, dtype=np.float64)
    nb = S["nbands"]
    bc = S["band_chunk"]
    lvl, req = S["lvl"], S["req"]
    # per band: its (chunk, level-in-chunk) steps in order
    steps = []
    for b in range(nb):
        st = []
        for c in range(bc[b], bc[b + 1]):
            for li in range(S["chunks"][c]["nl"]):
                st.append((c, li))
        steps.append(st)
    nxt = [0] * nb
    progress = [0] * nb
    window = [None] * nb
    wcol = [None] * nb
    staged = [None] * nb
    images = {}

    def level_reqs(c, li):
        """The requirements a level's kernel reads: the image's own list, or
        the global list where the image says so; checked against the
        global records."""
        I = images.get(c)
        if I is None:
            I = images[c] = _image(S, c)
        L = S["chunks"][c]["L0"] + li
        q0, nq = lvl[L, 0], lvl[L, 1]
        glob = req[q0:q0 + nq]
        assert bool(I["lv"][li, 3] & 1) == (nq > 0), "requirement flag disagrees"
        f, k = I["lq"][li]
        own = I["rq"][f:f + k] if k >= 0 else req[f:f + (-k - 1)]
        assert np.array_equal(own, glob), "image requirement list differs"
        return own

    def ready(b):
        c, li = steps[b][nxt[b]]
        return all(progress[r[0]] >= r[1] for r in level_reqs(c, li))

    left = sum(len(s) for s in steps)
    while left:
        b = next((bb for bb in range(nb - 1, -1, -1) if nxt[bb] < len(steps[bb]) and ready(bb)),
                 None)
        assert b is not None, "deadlock: no band can run its next level"
        if nxt[b] == 0:   # band start: window and staged first values
            window[b] = np.zeros((S["max_slots"] + 1, ld))
            wcol[b] = np.full(S["max_slots"] + 1, -1)
            staged[b] = {}
            for c in range(bc[b], bc[b + 1]):
                images[c] = _image(S, c)
                staged[b][c] = x[images[c]["xc"]].copy()
        c, li = steps[b][nxt[b]]
        I = images[c]
        row0, nrow = I["lv"][li, 0], I["lv"][li, 1]
        if nrow:
            ks = np.arange(row0, row0 + nrow)
            e0 = I["ri"][ks, 1] & 0xFFFF
            ne = I["ri"][ks, 1] >> 16
            E = np.concatenate([np.arange(s, s + n) for s, n in zip(e0, ne)])
            rid = np.repeat(np.arange(nrow), ne)
            col = I["ent"][E, 0]
            fl = I["ent"][E, 1]
            first = (fl & 1) != 0
            last = (fl & 2) != 0
            stg = (fl & 4) != 0
            slot = (fl >> 3) & 0xFFF
            xi = fl >> 15
            assert not np.any(stg & ~first)
            assert np.array_equal(I["xc"][xi[stg]], col[stg]), "staged value of another column"
            later = ~first
            assert np.all(slot[later] > 0) and np.array_equal(wcol[b][slot[later]], col[later]), \
                "window slot read for a column it does not hold"
            wr = slot > 0
            assert len(np.unique(col)) == len(col), "rows of one level share a column"
            vals = window[b][slot]
            fg = first & ~stg
            vals[fg] = x[col[fg]]
            vals[stg] = staged[b][c][xi[stg]]
            a = I["a"][E][:, None]
            coef = a - sh[None, :] * I["b"][E][:, None] if S["shifted"] else a
            acc = np.zeros((nrow, ld))
            np.add.at(acc, rid, coef * vals)
            r = np.zeros((nrow, ld)) if rhs is None else rhs[I["ri"][ks, 0]]
            if S["mode"] == 1:
                nrm = np.zeros((nrow, ld))
                np.add.at(nrm, rid, coef * coef)
                d = np.where(nrm > 0, (r - acc) / np.where(nrm > 0, nrm, 1.0), 0.0)
                cu = coef
            else:
                d = (r - acc) * I["inv"][ks][:, None]
                cu = a
            new = vals + d[rid] * cu
            window[b][slot[wr]] = new[wr]
            wcol[b][slot[wr]] = col[wr]
            x[col[last]] = new[last]
        nxt[b] += 1
        left -= 1
        L = S["chunks"][c]["L0"] + li
        publish = bool(I["lv"][li, 3] & 2)
        assert publish == bool(lvl[L, 2]), "publish flag disagrees"
        assert publish or nxt[b] < len(steps[b]), "a band's last level must publish"
        if publish:
            progress[b] = nxt[b]
    return x


def claim_model(S, ctas, order=None, handoff=2.0):
    """Completion time of a schedule in a model of the device: `ctas` CTAs
    claim bands in ticket order (`order`, default the schedule's own); a
    band holds its CTA from its claim to its last level; a level takes one
    unit and starts after the band's previous level and, for each
    requirement, `handoff` units after the required level ended."""
    import heapq
    nb = S["nbands"]
    order = [int(v) for v in (S["order"] if order is None else order)]
    bc, lvl, req = S["band_chunk"], S["lvl"], S["req"]
    fin = [None] * nb
    free = [0.0] * ctas
    for b in order:
        t = heapq.heappop(free)
        f = []
        if bc[b] < bc[b + 1]:
            L0 = S["chunks"][bc[b]]["L0"]
            last = S["chunks"][bc[b + 1] - 1]
            for L in range(L0, last["L0"] + last["nl"]):
                for bb, need in req[lvl[L, 0]:lvl[L, 0] + lvl[L, 1]]:
                    t = max(t, fin[int(bb)][int(need) - 1] + handoff)
                t += 1.0
                f.append(t)
        fin[b] = f
        heapq.heappush(free, t)
    return max(f[-1] for f in fin if f)
