"""APIC transfers with the conservative split (P2G) and merge (G2P).

TEST INFRASTRUCTURE ONLY (FP64 oracle).

P2G -- paper section "Transfer: P2G": grid mass and momentum from interior,
surface and balance particles with their split masses and the parent's v_p, A_p
(APIC splat v_p + A_p (x_i - x_*), x_* the particle's own position); grid
temperature from interior particles only with their full mass m_p.
Reading: the printed temperature transfer has no normalisation; the grid
temperature is the thermal-mass weighted average T_i = (sum m N (T + dT.(x_i - x_p))) / m^T_i
with m^T_i = sum_p m_p N_i(x_p).

G2P -- paper section "Transfer: G2P": merged momentum distribution
p_ip = m~_p v_i [N_i(x_p) + sum_{r in Pi_p} N_i(s_r) + N_i(b_r)],
v_p = sum_i p_ip / m_p, affine moments t_p = sum_i p_ip (x_i - x_p)^T and
A_p = 4 / (m_p dx^2) t_p (for Pi_p empty this is plain APIC G2P);
T_p = sum_i T_i N_i(x_p), grad T_p = sum_i T_i grad N_i(x_p).
"""
import numpy as np

from .spline import Stencil, scatter


def _apic_splat(st, mass, v, A):
    """mass N (v + A (x_i - x_*)) per stencil entry, (P, 27, 3)."""
    rel = st.xi - st.X[:, None, :]
    vel = v[:, None, :] + np.einsum("pab,pqb->pqa", A, rel)
    return (mass[:, None] * st.N)[:, :, None] * vel


def p2g(n, dx, x, v, A, mt, s=None, b=None, parent=None, m=None, T=None, gradT=None):
    """Grid mass, momentum and (optionally) thermal mass / temperature sums.

    Returns dict with m_i (G,), mv_i (G,3) and, when T is given, mT_i (G,) and
    mTT_i (G,) (the un-normalised mass-weighted temperature).
    """
    G = int(np.prod(n))
    st = Stencil(x, dx, n)
    mass = scatter(G, st.node, mt[:, None] * st.N)
    mom = scatter(G, st.node, _apic_splat(st, mt, v, A))
    if s is not None and s.shape[0]:
        for pos in (s, b):
            sp = Stencil(pos, dx, n)
            mp = mt[parent]
            mass += scatter(G, sp.node, mp[:, None] * sp.N)
            mom += scatter(G, sp.node, _apic_splat(sp, mp, v[parent], A[parent]))
    out = dict(m=mass, mv=mom)
    if T is not None:
        rel = st.xi - st.X[:, None, :]
        Tn = T[:, None] + np.einsum("pqa,pa->pq", rel, gradT)
        out["mT"] = scatter(G, st.node, m[:, None] * st.N)
        out["mTT"] = scatter(G, st.node, (m[:, None] * st.N) * Tn)
    return out


def grid_velocity(mass, mom):
    """v_i = (m v)_i / m_i on nodes with mass, zero elsewhere."""
    v = np.zeros_like(mom)
    act = mass > 0
    v[act] = mom[act] / mass[act, None]
    return v


def g2p(n, dx, vhat, x, m, mt, s=None, b=None, parent=None, That=None):
    """Merged G2P. Returns v_p, A_p and (when That is given) T_p, grad T_p."""
    G = int(np.prod(n))
    Np = x.shape[0]
    st = Stencil(x, dx, n)
    # per-particle momentum distribution on its own stencil nodes, plus the
    # group members' stencils; gather everything as (node, particle) pairs.
    nodes = [st.node]
    owners = [np.broadcast_to(np.arange(Np)[:, None], st.node.shape)]
    weights = [st.N]
    if s is not None and s.shape[0]:
        for pos in (s, b):
            sp = Stencil(pos, dx, n)
            nodes.append(sp.node)
            owners.append(np.broadcast_to(parent[:, None], sp.node.shape))
            weights.append(sp.N)
    node = np.concatenate([a.ravel() for a in nodes])
    owner = np.concatenate([a.ravel() for a in owners])
    w = np.concatenate([a.ravel() for a in weights])
    p_ip = (mt[owner] * w)[:, None] * vhat[node]                       # (K, 3)
    xi = (np.stack([node % n[0], (node // n[0]) % n[1], node // (n[0] * n[1])], -1) + 0.5) * dx
    r_ip = xi - x[owner]
    vp = np.zeros((Np, 3))
    tp = np.zeros((Np, 3, 3))
    for a in range(3):
        vp[:, a] = np.bincount(owner, weights=p_ip[:, a], minlength=Np)
        for c in range(3):
            tp[:, a, c] = np.bincount(owner, weights=p_ip[:, a] * r_ip[:, c], minlength=Np)
    vp /= m[:, None]
    Ap = tp * (4.0 / (m[:, None, None] * dx * dx))
    out = dict(v=vp, A=Ap, grad_v=np.einsum("pqa,pqb->pab", vhat[st.node], st.dN))
    if That is not None:
        out["T"] = np.einsum("pq,pq->p", st.N, That[st.node])
        out["gradT"] = np.einsum("pqa,pq->pa", st.dN, That[st.node])
    return out
