"""Dense complex linear algebra of the coupled subdomain system on the GPU (Section 3.5, steps
2(b)-(c)): the Householder QR, the triangular solves with its R, and the small matrix products
of the assembly, all by libmdp's kernels (mdp_householder_qr[_batched], mdp_triangular_solve,
mdp_complex_matmul). Argument marshalling only; CUDA complex128 tensors in, no host fallback."""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib


def _p(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need_cuda(*ts):
    for t in ts:
        if not (t.is_cuda and t.dtype == torch.complex128):
            raise TypeError("libmdp's dense linear algebra takes CUDA complex128 tensors")


def check_work(work, index, what):
    """Raise if the status word of a QR call (work[index], read after the stream) is not OK."""
    st = int(work[index].item())
    if st != _lib.MDP_OK:
        raise _lib.MdpError(st, what)


_pending = []   # (pinned host copy of status words, CUDA event after the copy) not yet checked


def defer_check(factor):
    """Queue the status words of a factor's QR launches for a later check_pending, without waiting
    for the stream: their copy to pinned host memory is enqueued behind the launches."""
    for work, index in factor.works:
        host = torch.empty(1, dtype=torch.int32, pin_memory=True)
        host.copy_(work[index:index + 1], non_blocking=True)
        ev = torch.cuda.Event()
        ev.record()
        _pending.append((host, ev))


def check_pending(wait=False):
    """Raise if a queued status word reports a device error. Without wait, only the copies that
    have completed are examined (the others stay queued)."""
    global _pending
    keep = []
    for host, ev in _pending:
        if wait:
            ev.synchronize()
        elif not ev.query():
            keep.append((host, ev))
            continue
        st = int(host[0])
        if st != _lib.MDP_OK:
            _pending = keep
            raise _lib.MdpError(st, "mdp_householder_qr (deferred status)")
    _pending = keep


class QRFactor:
    """An R factor of a tall m x n matrix A (R^H R = P^T A^H A P for the column order perm, the
    identity unless given) with qb = the first n entries of Q^H b in that order. F holds R
    column-major: R(i, j) = F[j, i] for i <= j, rows of ldr elements (entries below the diagonal
    are ignored). works: the status words of the QR launches behind it, (tensor, index) pairs."""

    def __init__(self, F, n, ldr, qb, works, perm=None):
        self.F, self.n, self.ldr, self.qb, self.works, self.perm = F, n, ldr, qb, works, perm

    def R(self):
        """R as a dense upper-triangular [n, n] tensor (in the column order perm)."""
        return torch.triu(self.F[:self.n, :self.n].transpose(0, 1))

    def check(self):
        """Raise if a QR launch behind this factor reported a device error (reads the status words:
        waits for the stream)."""
        for work, index in self.works:
            check_work(work, index, "mdp_householder_qr")

    def solve(self, rhs, conj_trans=False):
        """R^{-1} rhs (or R^{-H} rhs), in the column order perm: rhs [n] or [n, nrhs]."""
        return triangular_solve(self.F, self.n, self.ldr, rhs, conj_trans)

    def lstsq(self):
        """The least-squares solution x = argmin ||A x - b|| in A's own column order."""
        return self._unpermute(self.solve(self.qb))

    def gram_solve(self, g):
        """(A^H A)^{-1} g in A's own column order (two triangular solves)."""
        gp = g if self.perm is None else g[self.perm]
        return self._unpermute(self.solve(self.solve(gp, conj_trans=True)))

    def _unpermute(self, y):
        if self.perm is None:
            return y
        x = torch.empty_like(y)
        x[self.perm] = y
        return x


def triangular_solve(F, n, ldr, rhs, conj_trans=False):
    """X with R X = rhs (conj_trans: R^H X = rhs) for R the n x n upper triangle of the
    column-major factor F (R(i, j) = F[j, i]; F contiguous with rows of ldr elements)."""
    _need_cuda(F, rhs)
    if F.stride(-1) != 1 or F.stride(0) != ldr or rhs.shape[0] != n:
        raise ValueError("triangular_solve: F must hold rows of ldr contiguous elements and rhs n rows")
    vec = rhs.dim() == 1
    X = (rhs[:, None] if vec else rhs).transpose(0, 1).contiguous()   # [nrhs, n]: column-major n x nrhs
    _lib.check(_lib.lib().mdp_triangular_solve(n, X.shape[0], _p(F), ldr, int(bool(conj_trans)), _p(X), n, _stream()),
               "mdp_triangular_solve")
    return X[0] if vec else X.transpose(0, 1)


def _qr_launch(M, batch, m, n, ldm, stride):
    """mdp_householder_qr_batched on column-major blocks M with one right-hand side after the n
    columns; returns (tau, work)."""
    tau = torch.empty((batch, n), dtype=torch.complex128, device=M.device)
    work = torch.empty(int(_lib.lib().mdp_householder_qr_work_ints(batch)), dtype=torch.int32, device=M.device)
    _lib.check(_lib.lib().mdp_householder_qr_batched(batch, m, n, 1, _p(M), ldm, stride, _p(tau), _p(work),
                                                     _stream()),
               "mdp_householder_qr_batched")
    return tau, work


def householder_qr(A, b):
    """QRFactor of a tall complex CUDA matrix A [m, n] with right-hand side b [m] (one launch of
    mdp_householder_qr; .check() reads the device status)."""
    _need_cuda(A, b)
    m, n = A.shape
    M = torch.empty((n + 1, m), dtype=torch.complex128, device=A.device)   # column-major [A | b]
    M[:n] = A.transpose(0, 1)
    M[n] = b
    _, work = _qr_launch(M, 1, m, n, m, 0)
    return QRFactor(M, n, m, M[n, :n], [(work, 1)])


class _Structure:
    """The column split and the index tensors of a block-sparse least-squares structure (built once
    per structure and device: a host list turned into a device index is a synchronous copy)."""

    def __init__(self, n, rows, cols, dev):
        count = {}
        for cj in cols:
            for c in cj:
                count[c] = count.get(c, 0) + 1
        self.shared = sorted(c for c, v in count.items() if v > 1)
        self.private = [[c for c in cj if count[c] == 1] for cj in cols]
        self.order = [p + [c for c in cj if count[c] > 1] for p, cj in zip(self.private, cols)]   # private first
        self.mmax = max(rows)
        self.nmax = max(len(o) for o in self.order)
        self.ok = self.mmax >= self.nmax and sum(len(p) for p in self.private) + len(self.shared) == n
        self.npriv = n - len(self.shared)
        self.ns = len(self.shared)
        self.ms = sum(len(o) - len(p) for o, p in zip(self.order, self.private))
        self.ok = self.ok and (self.ns == 0 or self.ms >= self.ns)
        perm = [c for p in self.private for c in p] + self.shared
        pos = {c: i for i, c in enumerate(perm)}
        self.perm = torch.as_tensor(perm, device=dev)
        self.cidx = [torch.as_tensor(o, device=dev) for o in self.order]
        self.gidx = [torch.as_tensor([pos[c] for c in o], device=dev) for o in self.order]
        self.sidx = [torch.as_tensor([pos[c] - self.npriv for c in o[len(p):]], device=dev)
                     for o, p in zip(self.order, self.private)]


_structures = {}   # per (n, rows, cols, device); the least recently built go first beyond 32
_STRUCTURES_MAX = 32


def structured_qr(A, b, rows, cols):
    """QRFactor of A [m, n] whose row block j (rows[j] rows) has nonzeros only in the columns
    cols[j], by block elimination (a sparse QR in the nested-dissection order):
      1. a batched QR of every block on its own columns, those no other block touches (private)
         first: R_j = [[R_pp, R_ps], [0, R_ss]], Q_j^H b_j = [q_p; q_s];
      2. min sum_j ||R_pp x_p + R_ps x_s - q_p||^2 + ||R_ss x_s - q_s||^2 is met exactly in the
         private unknowns for any shared x_s, so one QR of the stacked R_ss (in the shared
         columns) with the stacked q_s gives R_s and q_s';
      3. R = [[R_pp,j ... R_ps,j], [0 ... R_s]] in the column order (private of block 0, ...,
         shared) is upper triangular with R^H R = P^T A^H A P, and qb = [q_p,j ...; q_s'].
    The minimiser and Gram matrix are those of one QR of A; the sequential chain is the block
    columns, then the shared columns, instead of all n columns."""
    _need_cuda(A, b)
    n = A.shape[1]
    batch = len(rows)
    dev = A.device
    key = (n, tuple(rows), tuple(tuple(c) for c in cols), str(dev))
    st = _structures.get(key)
    if st is None:
        if len(_structures) >= _STRUCTURES_MAX:
            _structures.pop(next(iter(_structures)))
        st = _structures[key] = _Structure(n, rows, cols, dev)
    if not st.ok:
        return householder_qr(A, b)
    mmax, nmax, npriv, ns, ms = st.mmax, st.nmax, st.npriv, st.ns, st.ms
    M = torch.zeros((batch, nmax + 1, mmax), dtype=torch.complex128, device=dev)   # column-major blocks
    r0 = 0
    for j, g in enumerate(rows):
        M[j, :len(st.order[j]), :g] = A[r0:r0 + g].index_select(1, st.cidx[j]).transpose(0, 1)
        M[j, nmax, :g] = b[r0:r0 + g]
        r0 += g
    _, work1 = _qr_launch(M, batch, mmax, nmax, mmax, (nmax + 1) * mmax)
    works = [(work1, batch)]
    F = torch.zeros((n, n), dtype=torch.complex128, device=dev)   # column-major R in the order perm
    qb = torch.empty(n, dtype=torch.complex128, device=dev)
    S = torch.zeros((ns + 1, max(ms, 1)), dtype=torch.complex128, device=dev)   # column-major [S | q_s]
    p0 = 0
    s0 = 0
    for j in range(batch):
        nj, pj_n = len(st.order[j]), len(st.private[j])
        Rj = M[j, :nj, :nj]                     # column-major: Rj[c, r] = R_j(r, c)
        if pj_n:
            # rows p0 .. p0+pj_n of R: R_pp and R_ps of block j, placed in their columns of the order perm
            blk = torch.zeros((n, pj_n), dtype=torch.complex128, device=dev)
            blk.index_copy_(0, st.gidx[j], torch.triu(Rj[:, :pj_n].transpose(0, 1)).transpose(0, 1))
            F[:, p0:p0 + pj_n] = blk
            qb[p0:p0 + pj_n] = M[j, nmax, :pj_n]
        sj = nj - pj_n
        if sj:
            Rss = torch.triu(Rj[pj_n:, pj_n:].transpose(0, 1))   # [sj, sj] row-major R_ss
            # blocks share columns but not rows: add, do not overwrite
            S[:ns].index_add_(0, st.sidx[j], torch.nn.functional.pad(Rss.transpose(0, 1), (s0, S.shape[1] - s0 - sj)))
            S[ns, s0:s0 + sj] = M[j, nmax, pj_n:nj]
        p0 += pj_n
        s0 += sj
    if ns:
        _, work2 = _qr_launch(S, 1, ms, ns, S.shape[1], 0)
        works.append((work2, 1))
        F[npriv:, npriv:] = torch.triu(S[:ns, :ns].transpose(0, 1)).transpose(0, 1)
        qb[npriv:] = S[ns, :ns]
    return QRFactor(F, n, n, qb, works, perm=st.perm)


class MatMul(torch.autograd.Function):
    """A @ B for complex128 CUDA tensors (A [m, k], B [k, n] or [k]) by mdp_complex_matmul, with
    its backward (grad_A = g B^H, grad_B = A^H g) by the same kernel."""

    @staticmethod
    def forward(ctx, A, B):
        ctx.save_for_backward(A, B)
        return _matmul(A, B)

    @staticmethod
    def backward(ctx, g):
        A, B = ctx.saved_tensors
        gA = gB = None
        if ctx.needs_input_grad[0]:
            gA = _matmul(g[:, None] if B.dim() == 1 else g, (B[None, :] if B.dim() == 1 else B.transpose(0, 1)),
                         conj_b=True)
        if ctx.needs_input_grad[1]:
            gB = _matmul(A.transpose(0, 1), g, conj_a=True)
        return gA, gB


def _matmul(A, B, conj_a=False, conj_b=False):
    """op(A) @ op(B) (op = conjugate if asked) for complex128 CUDA tensors given by their strides
    (a lazily conjugated view passes its data with the conjugation flag flipped)."""
    _need_cuda(A, B)
    if A.is_conj():
        A, conj_a = A.conj(), not conj_a
    if B.is_conj():
        B, conj_b = B.conj(), not conj_b
    vec = B.dim() == 1
    Bm = B[:, None] if vec else B
    m, k = A.shape
    if Bm.shape[0] != k:
        raise ValueError(f"matmul shapes {tuple(A.shape)} and {tuple(B.shape)}")
    n = Bm.shape[1]
    out = torch.empty((m, n), dtype=torch.complex128, device=A.device)
    _lib.check(_lib.lib().mdp_complex_matmul(m, n, k, _p(A), A.stride(0), A.stride(1), int(conj_a), _p(Bm),
                                             Bm.stride(0), Bm.stride(1), int(conj_b), _p(out), out.stride(0),
                                             out.stride(1), 0, _stream()),
               "mdp_complex_matmul")
    return out[:, 0] if vec else out


def matmul(A, B):
    """A @ B on libmdp's kernel, differentiable (MatMul); real operands are taken as complex."""
    if A.dtype != torch.complex128:
        A = A.to(torch.complex128)
    if B.dtype != torch.complex128:
        B = B.to(torch.complex128)
    return MatMul.apply(A, B)
