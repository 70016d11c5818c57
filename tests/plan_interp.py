"""CPU interpreter of the fused plan programs (GPU-path side, not the oracle).

It executes the forward and backward programs exported by qf_plan_export with
the same semantics as the pass kernels, but on whole complex128 state vectors,
so the planner's fusion, ordering, checkpoint placement, merged gradient terms
and reversal can be checked against the oracle without a GPU.
"""
from __future__ import annotations

import numpy as np

OP_STEP, OP_U, OP_G, OP_CHAIN, OP_CZ, OP_CKPT, OP_ANCHOR, OP_CNOT = 1, 2, 3, 4, 5, 6, 7, 8
SRC_GENERATE, BUF_WORK, BUF_NONE = -1, -2, -3
LAM_SEED, LAM_BUF = -1, -2
RX, RY, RZ = 0, 1, 2
FWD_ROUND_WORDS, BWD_ROUND_WORDS = 16, 12


class Program:
    pass


def _double(lo, hi):
    return float(np.array([lo & 0xFFFFFFFF, hi & 0xFFFFFFFF], np.uint32).view(np.float64)[0])


def parse(words):
    w = [int(v) for v in words]
    i = 0
    prog = Program()
    prog.rounds_mode = w[i] == 1
    i += 1
    prog.qshift = w[i]; i += 1  # circuit qubit q is simulated bit (q + qshift) mod n
    n_pass = w[i]; i += 1
    passes = []
    keys = ["op_begin", "op_end", "psi_src", "psi_dst", "lam_src", "lam_dst", "flags", "K", "n_groups",
            "outer_mask", "xm_local"]
    for _ in range(n_pass):
        d = dict(zip(keys, w[i:i + 11])); i += 11
        d["gmap"] = w[i:i + 16]; i += 16
        d["groups"] = [w[i + 4 * g:i + 4 * g + 4] for g in range(4)]; i += 16
        passes.append(d)
    n_ops = w[i]; i += 1
    prog.ops = [(w[i + 2 * k] & 0xFFFFFFFF, w[i + 2 * k + 1] & 0xFFFFFFFF) for k in range(n_ops)]
    i += 2 * n_ops
    nf = w[i]; i += 1
    prog.fused = []
    for _ in range(nf):
        cnt = w[i]; i += 1
        prog.fused.append([(w[i + 4 * j], w[i + 4 * j + 1], _double(w[i + 4 * j + 2], w[i + 4 * j + 3]))
                           for j in range(cnt)])
        i += 4 * cnt
    nr = w[i]; i += 1
    prog.round_words = w[i:i + nr]; i += nr
    nt = w[i]; i += 1
    prog.terms = []
    prog.term_const = []
    for _ in range(nt):
        kind, cnt = w[i], w[i + 1]
        prog.terms.append((kind, w[i + 2:i + 2 + cnt]))
        prog.term_const.append(_double(w[i + 2 + cnt], w[i + 3 + cnt]))
        i += 4 + cnt
    prog.passes = passes
    assert i == len(w)
    return prog


def rot(kind, t):
    c, s = np.cos(t / 2), np.sin(t / 2)
    if kind == RX:
        return np.array([[c, -1j * s], [-1j * s, c]])
    if kind == RY:
        return np.array([[c, -s], [s, c]], dtype=complex)
    return np.array([[c - 1j * s, 0], [0, c + 1j * s]])


PAULI = {RX: np.array([[0, 1], [1, 0]], complex), RY: np.array([[0, -1j], [1j, 0]]),
         RZ: np.array([[1, 0], [0, -1]], complex)}


def apply1(psi, n, q, u):
    v = psi.reshape(2 ** (n - 1 - q), 2, 2 ** q)
    return np.einsum("ab,xbz->xaz", u, v).reshape(-1)


def chain_sign(n, links):
    """Signs of the CZ links of a round: link q couples qubits q and q+1 mod n
    (link n-1 is a ring's CZ(n-1, 0))."""
    x = np.arange(2 ** n, dtype=np.int64)
    par = np.zeros(2 ** n, dtype=np.int64)
    for q in range(n):
        if (links >> q) & 1:
            par ^= ((x >> q) & 1) & ((x >> ((q + 1) % n)) & 1)
    return 1 - 2 * par


def cz_sign(n, c, t):
    x = np.arange(2 ** n, dtype=np.int64)
    return 1 - 2 * (((x >> c) & 1) & ((x >> t) & 1))


def cnot(psi, n, c, t):
    """Swap the amplitude pairs over bit t whose bit c is 1."""
    x = np.arange(2 ** n, dtype=np.int64)
    sel = (((x >> c) & 1) == 1) & (((x >> t) & 1) == 0)
    out = psi.copy()
    a, b = x[sel], x[sel] | (1 << t)
    out[a], out[b] = psi[b], psi[a]
    return out


def cnot_op(pd, group, w0, w1):
    """(control, target) global qubits of an OP_CNOT in pass pd."""
    t = pd["gmap"][group[(w0 >> 4) & 3]]
    c = pd["gmap"][group[w1 & 0xFF]] if (w1 >> 8) & 1 else (w1 & 0xFF)
    return c, t


def observable(psi, n, xm, zm):
    x = np.arange(2 ** n, dtype=np.int64)
    xp = x ^ xm
    ny = bin(xm & zm).count("1")
    par = np.array([bin(int(v) & zm).count("1") & 1 for v in xp])
    return (1j ** ny) * (1 - 2 * par) * psi[xp]


def encode(x, n, n_eff):
    psi = np.zeros(2 ** n_eff, complex)
    psi[0] = 1
    for q in range(n):
        psi = apply1(psi, n_eff, q, rot(RY, float(x[q])))
    return psi


def fused_matrix(prog, m, theta):
    u = np.eye(2, dtype=complex)
    for kind, p, angle in prog.fused[m]:
        u = rot(kind, float(theta[p]) if p >= 0 else angle) @ u
    return u


def term_angle(prog, t, theta):
    return float(sum(float(theta[p]) for p in prog.terms[t][1])) + prog.term_const[t]


def round_diagonal(n_eff, regs, phi, bbits, sign):
    """A round's RZ runs (angles phi[r] on qubits regs[r]) and its CZ links
    between register bits (bit r of bbits: regs[r], regs[r + 1]) as one
    diagonal over the whole vector, the way the round kernels apply it: the
    phase of register index j is exp(sign * i * a_j), a_j = sum_r sigma_r(j)
    phi_r / 2 with sigma_r(j) = +1 where bit r of j is clear (sign -1: the RZ
    runs applied, +1: un-applied), times -1 where a register-register link
    joins two set bits."""
    x = np.arange(2 ** n_eff, dtype=np.int64)
    j = np.zeros_like(x)
    for r in range(4):
        j |= ((x >> regs[r]) & 1) << r
    a = np.zeros(2 ** n_eff)
    for r in range(4):
        a += np.where((j >> r) & 1, -phi[r], phi[r]) / 2
    cz = np.zeros_like(x)
    for r in range(3):
        if (bbits >> r) & 1:
            cz ^= ((j >> r) & 1) & ((j >> (r + 1)) & 1)
    return np.exp(sign * 1j * a) * (1 - 2 * cz)


def _round_parts(prog, rec_tz, rec_ty, rx, regs, theta):
    phi = [term_angle(prog, t, theta) if t >= 0 else 0.0 for t in rec_tz]
    rots = []
    for r in range(4):
        t = rec_ty[r]
        if t >= 0:
            kind = RX if (rx >> r) & 1 else RY
            assert prog.terms[t][0] == kind
            rots.append((r, kind, term_angle(prog, t, theta)))
    return phi, rots


def _links_rest(links, bbits, regs):
    """The round's links other than those between register bits (those are in
    the diagonal table)."""
    for r in range(3):
        if (bbits >> r) & 1:
            assert regs[r + 1] == regs[r] + 1 and (links >> regs[r]) & 1
            links &= ~(1 << regs[r])
    return links


def fwd_ops(prog, pd, psi, n_eff, theta, slots, kernel_order=False):
    """Apply the forward op range of pass pd to psi (whole vector); OP_CKPT
    writes slots. kernel_order: round programs run as the round kernels do:
    the four rotations from the rotation terms, then the round's diagonal
    (its RZ-run terms and register-register CZ signs), then the other links;
    otherwise each item's fused 2x2 and then all the links."""
    k = pd["op_begin"]
    group = None
    while k < pd["op_end"]:
        w0, w1 = prog.ops[k]; k += 1
        code = w0 & 15
        if code == OP_STEP and prog.rounds_mode:
            group = pd["groups"][(w0 >> 4) & 3]
            nr = (w0 >> 8) & 0xFFFF
            for j in range(nr):
                rec = prog.round_words[(w1 + j) * FWD_ROUND_WORDS:(w1 + j + 1) * FWD_ROUND_WORDS]
                if kernel_order:
                    regs = [pd["gmap"][group[r]] for r in range(4)]
                    phi, rots = _round_parts(prog, rec[8:12], rec[12:16], rec[6], regs, theta)
                    for r, kind, angle in rots:
                        psi = apply1(psi, n_eff, regs[r], rot(kind, angle))
                    psi = psi * round_diagonal(n_eff, regs, phi, rec[5], -1)
                    psi = psi * chain_sign(n_eff, _links_rest(rec[4] & 0xFFFFFFFF, rec[5], regs))
                    continue
                for r in range(4):
                    psi = apply1(psi, n_eff, pd["gmap"][group[r]], fused_matrix(prog, rec[r], theta))
                psi = psi * chain_sign(n_eff, rec[4] & 0xFFFFFFFF)
        elif code == OP_STEP:
            group = pd["groups"][(w0 >> 4) & 3]
        elif code == OP_U:
            r, m = (w0 >> 4) & 3, w0 >> 8
            psi = apply1(psi, n_eff, pd["gmap"][group[r]], fused_matrix(prog, m, theta))
        elif code == OP_CHAIN:
            psi = psi * chain_sign(n_eff, w1)
        elif code == OP_CZ:
            psi = psi * cz_sign(n_eff, w1 & 255, (w1 >> 8) & 255)
        elif code == OP_CNOT:
            psi = cnot(psi, n_eff, *cnot_op(pd, group, w0, w1))
        elif code == OP_CKPT:
            slots[w1] = psi.copy()
        else:
            raise AssertionError(f"unexpected forward op {code}")
    return psi


def layout_mask(prog, m, n):
    """A mask of circuit qubits as simulated bits of the plan's layout."""
    s = getattr(prog, "qshift", 0)
    if s == 0:
        return m
    return ((m << s) | (m >> (n - s))) & ((1 << n) - 1)


def layout_x(prog, xrow, n):
    """Encoding angles per simulated bit: bit p holds circuit qubit (p - s) mod n."""
    s = getattr(prog, "qshift", 0)
    return np.asarray([xrow[(p - s) % n] for p in range(n)]) if s else xrow


def run_forward(prog, n, n_eff, theta, xrow, xm, zm, kernel_order=False):
    xrow, xm, zm = layout_x(prog, xrow, n), layout_mask(prog, xm, n), layout_mask(prog, zm, n)
    slots = {}
    work = None
    E = None
    for pd in prog.passes:
        src = pd["psi_src"]
        psi = encode(xrow, n, n_eff) if src == SRC_GENERATE else (slots[src] if src >= 0 else work).copy()
        psi = fwd_ops(prog, pd, psi, n_eff, theta, slots, kernel_order)
        dst = pd["psi_dst"]
        if dst >= 0:
            slots[dst] = psi.copy()
        elif dst == BUF_WORK:
            work = psi.copy()
        if pd["flags"] & 1:
            E = float(np.real(np.vdot(psi, observable(psi, n_eff, xm, zm))))
    return E, slots


def _grad_unapply(psi, lam, n_eff, q, kind, angle):
    g = 0.5 * np.imag(np.vdot(lam, apply1(psi, n_eff, q, PAULI[kind])))
    ud = rot(kind, angle).conj().T
    return g, apply1(psi, n_eff, q, ud), apply1(lam, n_eff, q, ud)


def bwd_ops(prog, pd, psi, lam, n_eff, theta, slots, grad_term, seen, kernel_order=False):
    """Run the adjoint op range of pass pd on (psi, lam); returns both.
    kernel_order: round programs run as the round kernels do: the other links,
    then the round's four RZ-run terms at once from Im(conj(lambda) psi) with
    the register signs, the diagonal un-applied from both states, then each
    rotation's term and un-apply."""
    k = pd["op_begin"]
    group = None
    while k < pd["op_end"]:
        w0, w1 = prog.ops[k]; k += 1
        code = w0 & 15
        if code == OP_STEP and prog.rounds_mode:
            group = pd["groups"][(w0 >> 4) & 3]
            nr = (w0 >> 8) & 0xFFFF
            for j in range(nr):
                rec = prog.round_words[(w1 + j) * BWD_ROUND_WORDS:(w1 + j + 1) * BWD_ROUND_WORDS]
                if kernel_order:
                    regs = [pd["gmap"][group[r]] for r in range(4)]
                    s = chain_sign(n_eff, _links_rest(rec[8] & 0xFFFFFFFF, rec[9], regs))
                    psi, lam = psi * s, lam * s
                    phi, rots = _round_parts(prog, rec[0:4], rec[4:8], rec[10], regs, theta)
                    w = np.imag(np.conj(lam) * psi)
                    x = np.arange(2 ** n_eff, dtype=np.int64)
                    for r in range(4):
                        t = rec[r]
                        if t >= 0:
                            grad_term[t] += 0.5 * np.sum(np.where((x >> regs[r]) & 1, -w, w))
                            seen[t] += 1
                    dg = round_diagonal(n_eff, regs, phi, rec[9], +1)
                    psi, lam = psi * dg, lam * dg
                    for r, kind, angle in rots:
                        g, psi, lam = _grad_unapply(psi, lam, n_eff, regs[r], kind, angle)
                        grad_term[rec[4 + r]] += g
                        seen[rec[4 + r]] += 1
                    continue
                s = chain_sign(n_eff, rec[8] & 0xFFFFFFFF)
                psi, lam = psi * s, lam * s
                for r in range(4):
                    q = pd["gmap"][group[r]]
                    for t in (rec[r], rec[4 + r]):
                        if t < 0:
                            continue
                        kind = prog.terms[t][0]
                        g, psi, lam = _grad_unapply(psi, lam, n_eff, q, kind, term_angle(prog, t, theta))
                        grad_term[t] += g
                        seen[t] += 1
        elif code == OP_STEP:
            group = pd["groups"][(w0 >> 4) & 3]
        elif code == OP_G:
            r, kind, t = (w0 >> 4) & 3, (w0 >> 6) & 3, w1
            assert kind == prog.terms[t][0]
            g, psi, lam = _grad_unapply(psi, lam, n_eff, pd["gmap"][group[r]], kind, term_angle(prog, t, theta))
            grad_term[t] += g
            seen[t] += 1
        elif code == OP_CHAIN:
            s = chain_sign(n_eff, w1)
            psi, lam = psi * s, lam * s
        elif code == OP_CZ:
            s = cz_sign(n_eff, w1 & 255, (w1 >> 8) & 255)
            psi, lam = psi * s, lam * s
        elif code == OP_CNOT:
            ct = cnot_op(pd, group, w0, w1)
            psi, lam = cnot(psi, n_eff, *ct), cnot(lam, n_eff, *ct)
        elif code == OP_ANCHOR:
            psi = slots[w1].copy()
        else:
            raise AssertionError(f"unexpected backward op {code}")
    return psi, lam


def _term_grad(prog, grad_term, seen, n_params):
    assert np.all(seen == 1), "every gradient term must appear exactly once"
    grad = np.zeros(n_params)
    for t, (_, params) in enumerate(prog.terms):
        for p in params:
            grad[p] += grad_term[t]
    return grad


def run_backward(prog, n_eff, theta, slots, xm, zm, dLdE, n_params, kernel_order=False):
    """Per-parameter gradient; every gradient term must be visited once."""
    xm, zm = layout_mask(prog, xm, n_eff), layout_mask(prog, zm, n_eff)  # a shift implies n = n_eff
    grad_term = np.zeros(len(prog.terms))
    seen = np.zeros(len(prog.terms), int)
    work = lam_buf = None
    for pd in prog.passes:
        src = pd["psi_src"]
        psi = (slots[src] if src >= 0 else work).copy()
        lam = 2 * dLdE * observable(psi, n_eff, xm, zm) if pd["lam_src"] == LAM_SEED else lam_buf.copy()
        psi, lam = bwd_ops(prog, pd, psi, lam, n_eff, theta, slots, grad_term, seen, kernel_order)
        if pd["psi_dst"] == BUF_WORK:
            work = psi
        if pd["lam_dst"] == LAM_BUF:
            lam_buf = lam
    return _term_grad(prog, grad_term, seen, n_params)


PF_SRC_H, PF_DST_H = 2, 4


def parse_schedule(words):
    """Mode A adjoint launch list (qf_plan_export direction 2)."""
    w = [int(v) for v in words]
    n = w[2]  # w[1]: the layout's qubit shift (as in the programs)
    keys = ["op_begin", "op_end", "psi_src", "psi_dst", "lam_src", "lam_dst", "flags", "K", "n_groups",
            "outer_mask", "xm_local"]
    out, i = [], 3
    for _ in range(n):
        d = dict(zip(keys, w[i + 1:i + 12]))
        d["dir"] = w[i]
        d["gmap"] = w[i + 12:i + 28]
        d["groups"] = [w[i + 28 + 4 * g:i + 32 + 4 * g] for g in range(4)]
        out.append(d)
        i += 44
    assert i == len(w)
    return out


def bf16_round(psi):
    """Round re and im to bfloat16 (nearest even), as the memory-saving store."""
    def r(v):
        b = np.asarray(v, np.float32).view(np.uint32).astype(np.uint64)
        b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
        return b.astype(np.uint32).view(np.float32).astype(np.float64)
    return r(psi.real) + 1j * r(psi.imag)


def run_backward_mode_a(fprog, bprog, sched, n, n_eff, theta, xrow, slots, xm, zm, dLdE, n_params):
    """Mode A: per block, forward segments re-run into pass-output slots, then
    adjoint segments from those stored outputs (psi never reversed across a
    segment boundary)."""
    grad_term = np.zeros(len(bprog.terms))
    seen = np.zeros(len(bprog.terms), int)
    aslots = {}
    lam_buf = None
    xrow, xm, zm = layout_x(bprog, xrow, n), layout_mask(bprog, xm, n), layout_mask(bprog, zm, n)

    def load(src, half):
        if src == SRC_GENERATE:
            return encode(xrow, n, n_eff)
        return (aslots[src] if half else slots[src]).copy()

    for pd in sched:
        half_src = bool(pd["flags"] & PF_SRC_H)
        if pd["dir"] == 0:
            psi = fwd_ops(fprog, pd, load(pd["psi_src"], half_src), n_eff, theta, {})
            if pd["flags"] & PF_DST_H:
                aslots[pd["psi_dst"]] = bf16_round(psi)
            else:
                slots[pd["psi_dst"]] = psi.copy()
        else:
            psi = load(pd["psi_src"], half_src)
            lam = 2 * dLdE * observable(psi, n_eff, xm, zm) if pd["lam_src"] == LAM_SEED else lam_buf.copy()
            psi, lam = bwd_ops(bprog, pd, psi, lam, n_eff, theta, slots, grad_term, seen)
            assert pd["psi_dst"] == BUF_NONE
            if pd["lam_dst"] == LAM_BUF:
                lam_buf = lam
    return _term_grad(bprog, grad_term, seen, n_params)
