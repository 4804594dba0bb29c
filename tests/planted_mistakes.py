"""Planted-mistake check of the oracle's pins and of the host builds of device code.

Plants one plausible mistake at a time in a copy of the oracle (a wrong sign, a
dropped term or factor, a transposed operand, a wrong threshold or tie rule) and
runs the oracle's pins against the copy; a pin suite that lets a mistake through
has a gap. Mistakes planted in the CUDA source (`dev_*`) are run against the
tests that build that source for the host and compare it with the oracle. The working tree is never modified: the repository's oracle, tests
and scene generators are copied to a temporary directory once, and each mistake
is applied to the copy and undone there.

Run by hand (it is not collected by pytest): python tests/planted_mistakes.py
[name ...]. About 40 s per mistake on one core. Each line reports CAUGHT or
SURVIVED with the last line of pytest's summary. A survivor is either a gap in
the pins or a change without effect (one is listed: `two_slip_not_fixed`; a node
with three slip walls is zeroed by the per-axis projection anyway).
"""
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# mistakes in the device source are checked by the host builds of that source
HOST = ["tests/test_mc_host.py", "tests/test_polar_host.py", "tests/test_surface_map_host.py",
        "tests/test_solid_map_host.py", "tests/test_cell_poly_host.py"]
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_surface.py", "tests/test_oracle_marching_cubes.py",
        "tests/test_scenes.py",
        "tests/test_golden.py::test_levelset_radius_is_the_papers_and_isolated_particles_cross_the_grid"]

# (name, file, text, replacement)
MISTAKES = [
    ('spline', 'oracle/spline.py', 'w = np.stack([0.5 * (1.5 - f) ** 2,', 'w = np.stack([0.5 * (1.5 - f) ** 2 * 1.0001,'),
    ('spline_dw_sign', 'oracle/spline.py', 'dw = np.stack([-(1.5 - f),', 'dw = np.stack([(1.5 - f),'),
    ('spline_xi_offset', 'oracle/spline.py', 'self.xi = (np.stack([ix, iy, iz], -1) + 0.5) * dx', 'self.xi = (np.stack([ix, iy, iz], -1) + 0.45) * dx'),
    ('balance_at_parent', 'oracle/resample.py', 'b = s + 2.0 * (x[parent] - s)', 'b = s + 1.0 * (x[parent] - s)'),
    ('split_mass', 'oracle/resample.py', 'mt = m / (2.0 * count + 1.0)', 'mt = m / (count + 1.0)'),
    ('apic_rel_sign', 'oracle/transfer.py', 'rel = st.xi - st.X[:, None, :]\n    vel', 'rel = st.X[:, None, :] - st.xi\n    vel'),
    ('g2p_A_factor', 'oracle/transfer.py', 'Ap = tp * (4.0 / (m[:, None, None] * dx * dx))', 'Ap = tp * (3.0 / (m[:, None, None] * dx * dx))'),
    ('g2p_no_balance', 'oracle/transfer.py', '        for pos in (s, b):\n            sp = Stencil(pos, dx, n)\n            nodes.append', '        for pos in (s,):\n            sp = Stencil(pos, dx, n)\n            nodes.append'),
    ('p2g_no_balance', 'oracle/transfer.py', '        for pos in (s, b):\n            sp = Stencil(pos, dx, n)\n            mp = mt[parent]', '        for pos in (s,):\n            sp = Stencil(pos, dx, n)\n            mp = mt[parent]'),
    ('temp_grad_sign', 'oracle/transfer.py', 'Tn = T[:, None] + np.einsum("pqa,pa->pq", rel, gradT)', 'Tn = T[:, None] - np.einsum("pqa,pa->pq", rel, gradT)'),
    ('J_no_dt', 'oracle/energy.py', 'J = (1.0 + dt * np.trace(Lp, axis1=1, axis2=2)) * self.Jn', 'J = (1.0 + np.trace(Lp, axis1=1, axis2=2)) * self.Jn'),
    ('liq_grad_no_Jn', 'oracle/energy.py', 'M = ((dt * self.lam_l * (J - 1.0) * self.Jn * self.V0) * liq)', 'M = ((dt * self.lam_l * (J - 1.0) * self.V0) * liq)'),
    ('visc_no_sym', 'oracle/energy.py', 'M = M + (dt * self.mu_l * self.Vn * liq)[:, None, None] * eps', 'M = M + (dt * self.mu_l * self.Vn * liq)[:, None, None] * Lp'),
    ('hess_liq_Jn1', 'oracle/energy.py', 'M = ((dt * dt * self.lam_l * self.Jn ** 2 * self.V0', 'M = ((dt * dt * self.lam_l * self.Jn * self.V0'),
    ('conformal_sign', 'oracle/energy.py', '+ (x12 - x21)[:, None, None]', '+ (x21 - x12)[:, None, None]'),
    ('surf_dn_no_proj', 'oracle/energy.py', 'dn = (dc - nrm * np.sum(nrm * dc, 1, keepdims=True)) / cn[:, None]', 'dn = dc / cn[:, None]'),
    ('surf_energy_no_gamma', 'oracle/energy.py', 'e_surf = np.sum(self.gamma * np.linalg.norm(c, axis=1))', 'e_surf = np.sum(np.linalg.norm(c, axis=1))'),
    ('fcr_P_cof', 'oracle/constitutive.py', '(lam * (J - 1.0))[:, None, None] * cof(F)\n', '(lam * (J - 1.0))[:, None, None] * F\n'),
    ('fcr_dR_sign', 'oracle/constitutive.py', '(2.0 * mu[:, None, None] * (dF - dR)', '(2.0 * mu[:, None, None] * (dF + dR)'),
    ('heat_robin_sign', 'oracle/heat.py', 'out += scatter(self.G, ss.node, (self.h * self.area * Ts)[:, None] * self.wS)', 'out -= scatter(self.G, ss.node, (self.h * self.area * Ts)[:, None] * self.wS)'),
    ('heat_source_N', 'oracle/heat.py', 'out += scatter(self.G, st.node, (self.H * self.Vn)[:, None] * st.N)', 'out += scatter(self.G, st.node, (self.H * self.Vn)[:, None] * st.N * 0.5)'),
    ('heat_no_K', 'oracle/heat.py', '(self.K * self.Vn)[:, None]', '(self.Vn)[:, None]'),
    ('newton_init', 'oracle/solver.py', 'v = proj(state.vn + prm.dt * state.g)', 'v = proj(state.vn)'),
    ('armijo_sign', 'oracle/solver.py', 'if phi(alpha) <= phi0 + c * alpha * slope:', 'if phi(alpha) <= phi0 - c * alpha * slope:'),
    ('final_force_eval', 'oracle/solver.py', '    v = v - r * inv_m[:, None]\n', '    v = v\n'),
    ('g2p_J_trace', 'oracle/step.py', 'sc.J = np.where(liq, (1.0 + dt * np.trace(Lg, axis1=1, axis2=2)) * sc.J, sc.J)', 'sc.J = np.where(liq, (1.0 - dt * np.trace(Lg, axis1=1, axis2=2)) * sc.J, sc.J)'),
    ('advect', 'oracle/step.py', 'sc.x = sc.x + dt * sc.v', 'sc.x = sc.x + 0.5 * dt * sc.v'),
    ('carry_dA_transpose', 'oracle/step.py', 'sc.dA = np.einsum("rab,rb->ra", cof(np.eye(3) + dt * Ls), sc.dA)', 'sc.dA = np.einsum("rba,rb->ra", cof(np.eye(3) + dt * Ls), sc.dA)'),
    ('wall_layers', 'oracle/boundary.py', 'on = (idx[axis] <= 1) if side == 0 else (idx[axis] >= n[axis] - 2)', 'on = (idx[axis] <= 0) if side == 0 else (idx[axis] >= n[axis] - 2)'),
    ('plane_below_sign', 'oracle/boundary.py', '        on_plane = phi < 0\n', '        on_plane = phi > 0\n'),
    ('slip_keeps_normal', 'oracle/boundary.py', '        P[sel] = np.eye(3) - np.outer(nn, nn)', '        P[sel] = np.eye(3) - 0.5 * np.outer(nn, nn)'),
    ('two_slip_not_fixed', 'oracle/boundary.py', '            | (nslip == 3))', '            )'),
    ('heat_rhs_b', 'oracle/heat.py', '((self.h * self.Tbar + self.b) * self.area)', '((self.h * self.Tbar) * self.area)'),
    ('heat_no_renorm', 'oracle/heat.py', 'self.wS = np.where(tot > 0, w / np.where(tot > 0, tot, 1.0), 0.0)', 'self.wS = w'),
    ('heat_diag_dt', 'oracle/heat.py', 'self.diag = cp * mT / dt', 'self.diag = cp * mT'),
    ('gamma_slope_sign', 'oracle/step.py', 'g = np.clip(g0 + g1 * (T - prm.T0), gmin, gmax)', 'g = np.clip(g0 - g1 * (T - prm.T0), gmin, gmax)'),
    ('gamma_sl_ignored', 'oracle/step.py', 'return np.where(kind == 1, prm.gamma_sl, g)', 'return g'),
    ('gamma_T_unnormalised', 'oracle/step.py', 'np.sum(ss.N * has * self.Tn[ss.node], 1) / np.where(wsum > 0, wsum, 1.0)', 'np.sum(ss.N * has * self.Tn[ss.node], 1)'),
    ('youngs_shape', 'oracle/step.py', 'prm.E0 * np.maximum(0.0, (prm.T_melt - T) / (prm.T_melt - prm.T0))', 'prm.E0 * np.maximum(0.0, (prm.T_melt - T) / (prm.T_melt))'),
    ('solid_lame_nu', 'oracle/step.py', 'youngs(T, prm) / (2.0 * (1.0 + prm.nu))', 'youngs(T, prm) / (2.0 * (1.0 - prm.nu))'),
    ('levelset_r0', 'oracle/surface.py', 'R0_FACTOR = 0.867', 'R0_FACTOR = 0.8'),
    ('sample_weight', 'oracle/surface.py', 'w = 1.0 / (nn * density)', 'w = 0.5 / (nn * density)'),
    ('osada_sqrt', 'oracle/surface.py', 'a = math.sqrt(r1)', 'a = r1'),
    ('kind_threshold', 'oracle/surface.py', 'kind = np.where(s @ np.asarray(pn, np.float64) - pd < dx, 1, 0)', 'kind = np.where(s @ np.asarray(pn, np.float64) - pd < 0.5 * dx, 1, 0)'),
    ('kinetic_half', 'oracle/energy.py', 'kin = 0.5 * np.sum(self.m[a] * np.sum(dv[a] ** 2, -1))', 'kin = np.sum(self.m[a] * np.sum(dv[a] ** 2, -1))'),
    ('gravity_sign', 'oracle/energy.py', '- dt * np.sum(self.m[a] * (v[a] @ self.g))', '+ dt * np.sum(self.m[a] * (v[a] @ self.g))'),
    ('visc_weight_V0', 'oracle/energy.py', 'self.Vn = np.where(self.liq, Jn, detF) * V0', 'self.Vn = V0'),
    ('solid_F_order', 'oracle/energy.py', 'F = np.einsum("pab,pbc->pac", np.eye(3) + dt * Lp, self.Fn)', 'F = np.einsum("pab,pbc->pac", self.Fn, np.eye(3) + dt * Lp)'),
    ('surface_C_transpose', 'oracle/energy.py', 'return np.einsum("agk,bdl,rb,rkl->ragd", EPS, EPS, self.dA, Fh)', 'return np.einsum("agk,bdl,rb,rlk->ragd", EPS, EPS, self.dA, Fh)'),
    ('nearest_ties', 'oracle/resample.py', 'out[lo:lo + chunk] = np.argmin(dist, axis=1)', 'out[lo:lo + chunk] = dist.shape[1] - 1 - np.argmin(dist[:, ::-1], axis=1)'),
    ('g2p_T_grad', 'oracle/transfer.py', 'out["gradT"] = np.einsum("pqa,pq->pa", st.dN, That[st.node])', 'out["gradT"] = 0.5 * np.einsum("pqa,pq->pa", st.dN, That[st.node])'),
    ('p2g_thermal_mass_split', 'oracle/transfer.py', 'out["mT"] = scatter(G, st.node, m[:, None] * st.N)', 'out["mT"] = scatter(G, st.node, mt[:, None] * st.N)'),
    ('friction_half', 'oracle/boundary.py', '    lim = -mu * vn[sel]', '    lim = -0.5 * mu * vn[sel]'),
    ('node_pos_offset', 'oracle/spline.py', 'return (np.stack([i.ravel(), j.ravel(), k.ravel()], -1) + 0.5) * dx', 'return (np.stack([i.ravel(), j.ravel(), k.ravel()], -1) + 0.25) * dx'),
    ('hess_visc_nosym', 'oracle/energy.py', '* 0.5 * (dL + np.swapaxes(dL, 1, 2))', '* dL'),
    ('surf_grad_sign', 'oracle/energy.py', 'Gs = self.gamma[:, None, None] * np.einsum', 'Gs = -self.gamma[:, None, None] * np.einsum'),
    ('robin_scatter_N', 'oracle/heat.py', 'out += scatter(self.G, ss.node, (self.h * self.area * Ts)[:, None] * self.wS)', 'out += scatter(self.G, ss.node, (self.h * self.area * Ts)[:, None] * self.ss.N)'),
    ('g2p_v_by_mt', 'oracle/transfer.py', '    vp /= m[:, None]', '    vp /= mt[:, None]'),
    ('fcr_mu_lam_swap', 'oracle/constitutive.py', 'return mu * np.sum((sig - 1.0) ** 2, -1) + 0.5 * lam * (J - 1.0) ** 2', 'return lam * np.sum((sig - 1.0) ** 2, -1) + 0.5 * mu * (J - 1.0) ** 2'),
    ('polar_sign_fix', 'oracle/constitutive.py', '    sig[dU, 2] *= -1.0\n', '\n'),
    ('cof_half', 'oracle/constitutive.py', 'return 0.5 * np.einsum("agk,bdl,...gd,...kl->...ab", EPS, EPS, F, F)', 'return np.einsum("agk,bdl,...gd,...kl->...ab", EPS, EPS, F, F)'),
    ('sticky_plane_slip', 'oracle/boundary.py', '        if plane_mode == 2:\n            sticky |= on_plane', '        if plane_mode == 3:\n            sticky |= on_plane'),
    ('sphere_outside_flip', 'oracle/boundary.py', '    R, outside = float(sphere[3]), bool(sphere[4])', '    R, outside = float(sphere[3]), not bool(sphere[4])'),
    ('heat_Vn_source', 'oracle/step.py', 'Vn = np.where(sc.phase == 0, sc.J, np.linalg.det(sc.F)) * sc.V0', 'Vn = sc.V0'),
    ('tet_orientation', 'oracle/surface.py', 'if (nrm[0] * g[0] + nrm[1] * g[1]) + nrm[2] * g[2] < 0.0:', 'if (nrm[0] * g[0] + nrm[1] * g[1]) + nrm[2] * g[2] > 0.0:'),
    ('mc_decider', 'oracle/surface.py', 'joined = cphi[ins[0]] * cphi[ins[1]] > cphi[out[0]] * cphi[out[1]]', 'joined = cphi[ins[0]] * cphi[ins[1]] < cphi[out[0]] * cphi[out[1]]'),
    ('mc_face_order', 'oracle/surface.py', 'uv = ((0, 0), (1, 0), (1, 1), (0, 1)) if s == 1 else ((0, 0), (0, 1), (1, 1), (1, 0))', 'uv = ((0, 0), (1, 0), (1, 1), (0, 1))'),
    ('poisson_mean', 'oracle/surface.py', 'lam = density * area', 'lam = 0.5 * density * area'),
    ('poisson_recursion', 'oracle/surface.py', 'p = p * lam / k', 'p = p * lam / (k + 1)'),
    ('levelset_clamp', 'oracle/surface.py', 'phi = np.minimum(dd, CLAMP_FACTOR * dx) - r0', 'phi = np.minimum(dd, 1.0 * dx) - r0'),
    ('melt_threshold', 'oracle/step.py', 'melt = (sc.phase == 1) & (sc.T > prm.T_melt)', 'melt = (sc.phase == 1) & (sc.T > prm.T_melt + 1.0)'),
    ('freeze_never', 'oracle/step.py', 'freeze = (sc.phase == 0) & (sc.T < prm.T_melt)', 'freeze = (sc.phase == 0) & (sc.T < prm.T0 - 1e9)'),
    ('gamma_clamp', 'oracle/step.py', 'g = np.clip(g0 + g1 * (T - prm.T0), gmin, gmax)', 'g = g0 + g1 * (T - prm.T0)'),
    ('grid_T_unnormalised', 'oracle/step.py', 'self.Tn = np.where(mT > 0, out["mTT"] / np.where(mT > 0, mT, 1.0), 0.0)', 'self.Tn = np.where(mT > 0, out["mTT"], 0.0)'),
    ('friction_stop', 'oracle/boundary.py', 's = np.where(tl > lim, 1.0 - lim / np.where(tl > 0, tl, 1.0), 0.0)', 's = np.where(tl > lim, 1.0 - lim / np.where(tl > 0, tl, 1.0), 1.0)'),
    ('friction_plane_normal', 'oracle/step.py', 'normals[on_p] = nn / np.linalg.norm(nn)', 'normals[on_p] = -nn / np.linalg.norm(nn)'),
    ('sphere_kind_band', 'oracle/step.py', 'near |= sphere_phi_normal(sc.s, sc.sphere)[0] < sc.dx', 'near |= sphere_phi_normal(sc.s, sc.sphere)[0] < 0.5 * sc.dx'),
    ('friction_sphere_normal', 'oracle/step.py', 'normals[on_s] = sphere_phi_normal(node_positions(sc.n, sc.dx)[on_s], sc.sphere)[1]', 'normals[on_s] = -sphere_phi_normal(node_positions(sc.n, sc.dx)[on_s], sc.sphere)[1]'),
    ('friction_drops_normal', 'oracle/boundary.py', 'out[sel] = s[:, None] * t + vn[sel, None] * nsel', 'out[sel] = s[:, None] * t'),
    ('fixed_nodes_free', 'oracle/boundary.py', '    P[full] = 0.0\n', '\n'),
    ('osada_b1', 'oracle/surface.py', 'b1 = a * (1.0 - r2)', 'b1 = (1.0 - r2)'),
    ('kmax', 'oracle/surface.py', 'KMAX = 31', 'KMAX = 3'),
    ('cube_range', 'oracle/surface.py', 'if min(m) >= 0 and m[0] < n[0] - 1 and m[1] < n[1] - 1 and m[2] < n[2] - 1:', 'if min(m) >= 1 and m[0] < n[0] - 1 and m[1] < n[1] - 1 and m[2] < n[2] - 1:'),
    ('dev_mc_decider', 'paper_2101_12408_gb300/csrc/mcubes.cuh', 'const bool joined = rmul(cphi[fc[i0]], cphi[fc[i0 + 2]]) > rmul(', 'const bool joined = rmul(cphi[fc[i0]], cphi[fc[i0 + 2]]) < rmul('),
    ('dev_mc_pairing', 'paper_2101_12408_gb300/csrc/mcubes.cuh', '(joined ? ce[(k + 3) & 3] : ce[(k + 1) & 3])', '(joined ? ce[(k + 1) & 3] : ce[(k + 3) & 3])'),
    ('dev_mc_face_order', 'paper_2101_12408_gb300/csrc/mcubes.cuh', 'const int iu = s ? (k == 1 || k == 2) : (k >= 2);', 'const int iu = (k == 1 || k == 2);'),
    ('dev_polar_cross', 'paper_2101_12408_gb300/csrc/polar.cuh', 'u[2][0] = u[0][1] * u[1][2] - u[0][2] * u[1][1];', 'u[2][0] = u[0][2] * u[1][1] - u[0][1] * u[1][2];'),
    ('dev_polar_sort', 'paper_2101_12408_gb300/csrc/polar.cuh', 'if (lam[0] < lam[1]) swap_cols(V, lam, 0, 1);', ''),
    ('dev_polar_kinv', 'paper_2101_12408_gb300/csrc/polar.cuh', 'R e[3] = {sig[1] + sig[2], sig[0] + sig[2], sig[0] + sig[1]};', 'R e[3] = {sig[0] + sig[2], sig[1] + sig[2], sig[0] + sig[1]};'),
    ('dev_fcr_dR_sign', 'paper_2101_12408_gb300/csrc/polar.cuh', 'dP[k] = R(2) * mu * (dF[k] - dR[k])', 'dP[k] = R(2) * mu * (dF[k] + dR[k])'),
    ('dev_surf_conformal', 'paper_2101_12408_gb300/csrc/newton.cu', 'R q = R(0.5) * k * an * (x12 - x21);', 'R q = R(0.5) * k * an * (x21 - x12);'),
    ('dev_surf_dn', 'paper_2101_12408_gb300/csrc/newton.cu', '        R dn[3] = {(dc[0] - nd * nv[0]) * ic', '        R dn[3] = {(dc[0]) * ic'),
    ('dev_frame_hand', 'paper_2101_12408_gb300/csrc/newton.cu', 't2[0] = u[1] * t1[2] - u[2] * t1[1];', 't2[0] = -(u[1] * t1[2] - u[2] * t1[1]);'),
    ('dev_solid_twist', 'paper_2101_12408_gb300/csrc/newton.cu', 'lv = R(2) * mu - R(4) * mu / den + lam * (J - R(1)) * s[z];', 'lv = R(2) * mu + R(4) * mu / den + lam * (J - R(1)) * s[z];'),
    ('dev_solid_pair', 'paper_2101_12408_gb300/csrc/newton.cu', 'lv = R(2) * mu - lam * (J - R(1)) * s[z];', 'lv = R(2) * mu + lam * (J - R(1)) * s[z];'),
    ('dev_solid_clamp', 'paper_2101_12408_gb300/csrc/newton.cu', 'if (!(lv > R(0))) continue;', ''),
    ('dev_solid_W', 'paper_2101_12408_gb300/csrc/newton.cu', 'matmul3_bt<R>(Qm, Fo, W);', 'matmul3<R>(Qm, Fo, W);'),
    ('dev_wT', 'paper_2101_12408_gb300/csrc/newton.cu', 'o2 = R(0.5) * (v0 + v2) - v1;', 'o2 = R(0.5) * (v0 + v2) + v1;'),
    ('dev_dT', 'paper_2101_12408_gb300/csrc/newton.cu', 'o1 = v0 - R(2) * v1 + v2;', 'o1 = v0 - R(2) * v1 - v2;'),
    ('dev_wN', 'paper_2101_12408_gb300/csrc/newton.cu', 'n0 = R(0.5) * (m0 + m2) - m1;', 'n0 = R(0.5) * (m0 + m2) + m1;'),
    ('dev_dN', 'paper_2101_12408_gb300/csrc/newton.cu', 'n1 = m0 - R(2) * m1;', 'n1 = m0 + R(2) * m1;'),
    ('dev_pair_middle', 'paper_2101_12408_gb300/csrc/newton.cu', 'const V p12 = P::make(p01.y, p23.x);', 'const V p12 = P::make(p01.x, p23.y);'),
    ('dev_pdN', 'paper_2101_12408_gb300/csrc/newton.cu', 'n1 = vfma(m1, m2, m0);', 'n1 = vfma(m0, m2, m1);'),
    ('dev_pair_rows', 'paper_2101_12408_gb300/csrc/newton.cu', 'lo[b][c] = P::make(n0.x, n1.x + n0.y);', 'lo[b][c] = P::make(n0.x, n1.x);'),
    ('dev_sample_exact_curv', 'paper_2101_12408_gb300/csrc/newton.cu', 'surf_G<R>(k * dt * dt, nv, dFh, av, G2);', 'surf_G<R>(k * dt * dt, nv, Fh, av, G2);'),
]


def _copy_tree(dst):
    for d in ("oracle", "tests", "paper_2101_12408_gb300", "include"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(dst, d),
                        ignore=shutil.ignore_patterns("_build", "*.so", "*.o", "__pycache__"))
    # the pins import the binding package's scene generators only; its library is not needed
    with open(os.path.join(dst, "tests", "conftest.py"), "w") as fh:
        fh.write("import os, sys\n"
                 "ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))\n"
                 "sys.path.insert(0, ROOT)\n"
                 "def pytest_configure(config):\n"
                 "    config.addinivalue_line('markers', 'gpu: needs a GPU')\n"
                 "    config.addinivalue_line('markers', 'slow: long CPU test')\n")


def main(names):
    with tempfile.TemporaryDirectory() as tmp:
        _copy_tree(tmp)
        for name, rel, text, repl in MISTAKES:
            if names and name not in names:
                continue
            path = os.path.join(tmp, rel)
            with open(path) as fh:
                src = fh.read()
            if text not in src:
                print(f"{name:24s} NOT FOUND (the source changed)", flush=True)
                continue
            with open(path, "w") as fh:
                fh.write(src.replace(text, repl, 1))
            try:
                tests = HOST if "/csrc/" in rel else PINS
                r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                                    "-m", "not gpu"] + tests, capture_output=True, text=True, cwd=tmp, timeout=900)
                out = r.stdout.strip().splitlines()
                print(f"{name:24s} {'CAUGHT' if r.returncode else 'SURVIVED'}  {out[-1] if out else ''}", flush=True)
            finally:
                with open(path, "w") as fh:
                    fh.write(src)


if __name__ == "__main__":
    main(set(sys.argv[1:]))
