"""PDHG with PDLP's adaptive steps, restarts and termination (oracle; test infrastructure).

Iteration (Sec. II.E, read in the general form of ``oracle.lp``), in the
rescaled space of ``oracle.scaling``, with step eta and primal weight omega,
tau = eta / omega and sigma = eta * omega:

  x+ = proj_[l, u]( x - tau (c - K^T y) )                      (primal step)
  y+ = proj_[y_lo, inf)( y + sigma (q - K (2 x+ - x)) )        (dual step)

The paper cites Applegate et al. for adaptive step sizes and restarts without
stating them (Sec. II.E).  Readings used here (the GPU solver follows the same
ones; its code shares nothing with this file):

* step rule: with dx = x+ - x, dy = y+ - y and k the 1-based count of step
  attempts so far,
      eta_max = (omega ||dx||^2 + ||dy||^2 / omega) / (2 |dy^T K dx|)   (inf if 0)
      eta'    = min((1 - (k+1)^-0.3) eta_max, (1 + (k+1)^-0.6) eta)
  the attempt is accepted iff eta <= eta_max; either way eta <- eta'.
  eta_0 = 1 / max|K~_ij|;  omega_0 = ||c~|| / ||q~|| (1 if either < 1e-10).
* averages: step-size weighted averages of accepted iterates since the last
  restart.
* every ``check_every`` attempts: rel-KKT (``oracle.lp``) of the current and the
  average iterate on the unscaled LP; stop when either is <= tol (the smaller
  wins).  Restart candidate = the one with smaller
      KKT_omega = sqrt(omega ||r~_p||^2 + ||r~_d||^2 / omega + (P - D)^2)
  (scaled residuals).  Restart iff KKT_omega(cand) <= 0.2 KKT_0, or
  (<= 0.8 KKT_0 and > the previous check's value), or the attempts since the
  last restart are >= 0.36 of all attempts.  On restart, with
  Dx = ||x_cand - x_anchor||, Dy = ||y_cand - y_anchor||, if both > 1e-10:
      omega <- exp(0.5 log(Dy / Dx) + 0.5 log omega)
  the iterate, anchor and KKT_0 move to the candidate (KKT_0 taken with the
  new omega, which also becomes the "previous" value) and the averages reset.

* infeasibility (Applegate et al.'s detection from iterate differences): at
  every check after the optimality test, the differences since the last
  restart of the current iterate and of the average, (x_c - x_anchor,
  y_c - y_anchor) taken back to the unscaled LP, are tested as rays
  (``oracle.lp.ray_check``): a dual ray with positive objective and violation
  <= eps_infeasible x objective proves primal infeasibility, a primal ray with
  negative cost and violation <= eps_infeasible x |cost| dual infeasibility
  (status "primal_infeasible" / "dual_infeasible"); eps_infeasible = 1e-8.

``schedule`` replays a recorded run: per attempt (eta, accepted) and per check
(restart, to_average); the oracle then follows those decisions while still
computing and returning its own, so that both can be compared.  The primal
weight is never replayed: it is always the oracle's own, updated at each
restart from the oracle's own iterates, so a replay compares the primal-weight
update too.  (The step size is replayed because the GPU evaluates the factors
(k+1)^-0.3 and (k+1)^-0.6 in FP32; the oracle's own eta_next is logged beside.)

The three rules are separate functions (``step_size_update``,
``restart_decision``, ``primal_weight_update``) so that each can be checked by
hand on its own.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .lp import LP, kkt, project_reduced_cost, ray_check
from .scaling import rescale


@dataclass
class PDLPOptions:
    check_every: int = 64
    beta_sufficient: float = 0.2
    beta_necessary: float = 0.8
    beta_artificial: float = 0.36
    omega_smoothing: float = 0.5
    step_reduction_exp: float = 0.3
    step_growth_exp: float = 0.6
    ruiz_iters: int = 10
    pock_chambolle: bool = True
    eps_infeasible: float = 1e-8  # 0 disables the infeasibility test


@dataclass
class PDHGResult:
    x: np.ndarray            # unscaled primal
    y: np.ndarray            # unscaled dual
    x_scaled: np.ndarray
    y_scaled: np.ndarray
    status: str
    attempts: int
    accepted: int
    restarts: int
    rel_kkt: float
    primal_obj: float
    dual_obj: float
    eta: float
    omega: float
    Dr: np.ndarray
    Dc: np.ndarray
    attempt_log: list = field(default_factory=list)  # (eta, omega, accepted, eta_max)
    check_log: list = field(default_factory=list)    # dict per check
    x_cur: np.ndarray | None = None   # unscaled current iterate at exit
    y_cur: np.ndarray | None = None
    x_avg: np.ndarray | None = None   # unscaled average since the last restart at exit
    y_avg: np.ndarray | None = None


def step_size_update(eta: float, omega: float, dx: np.ndarray, dy: np.ndarray, Kdx: np.ndarray, k: int,
                     opts: PDLPOptions):
    """Adaptive step rule of attempt k (1-based count of attempts so far) with
    dx = x+ - x, dy = y+ - y, Kdx = K dx.  Returns (accept, eta_max, eta_next)."""
    movement = omega * float(dx @ dx) + float(dy @ dy) / omega
    interaction = 2.0 * abs(float(dy @ Kdx))
    eta_max = movement / interaction if interaction > 0 else np.inf
    eta_next = min((1.0 - (k + 1) ** (-opts.step_reduction_exp)) * eta_max,
                   (1.0 + (k + 1) ** (-opts.step_growth_exp)) * eta)
    return eta <= eta_max, eta_max, eta_next


def restart_decision(kkt_cur: float, kkt_avg: float, has_avg: bool, kkt0: float, kkt_prev: float,
                     since_restart: int, attempts: int, opts: PDLPOptions):
    """Restart test at a check.  The candidate is the average when it has a
    smaller KKT_omega than the current iterate.  Returns (restart, to_avg, kkt_cand)."""
    to_avg = bool(has_avg and kkt_avg < kkt_cur)
    kc = kkt_avg if to_avg else kkt_cur
    restart = (kc <= opts.beta_sufficient * kkt0) or \
              (kc <= opts.beta_necessary * kkt0 and kc > kkt_prev) or \
              (since_restart >= opts.beta_artificial * attempts)
    return bool(restart), to_avg, kc


def primal_weight_update(omega: float, dist_x: float, dist_y: float, theta: float) -> float:
    """Primal weight after a restart that moved the primal iterate by dist_x and
    the dual by dist_y since the previous restart (log-space smoothing theta);
    unchanged when either distance is below 1e-10."""
    if dist_x > 1e-10 and dist_y > 1e-10:
        return float(np.exp(theta * np.log(dist_y / dist_x) + (1.0 - theta) * np.log(omega)))
    return omega


def _kkt_omega(slp: LP, Dr, Dc, lp: LP, x_s, y_s, omega):
    """Scaled-space restart metric and unscaled rel-KKT of one candidate."""
    res = kkt(lp, Dc * x_s, Dr * y_s)
    rp_s = Dr * res.rp
    rd_s = Dc * res.rd
    gap = res.primal_obj - res.dual_obj
    val = np.sqrt(omega * (rp_s @ rp_s) + (rd_s @ rd_s) / omega + gap * gap)
    return float(val), res


def pdhg_solve(lp: LP, tol: float = 1e-8, max_attempts: int = 1_000_000, opts: PDLPOptions | None = None,
               schedule: dict | None = None, fixed: dict | None = None, record: bool = False,
               stop_after: int | None = None, start: tuple | None = None, on_check=None) -> PDHGResult:
    """Solve ``lp`` to rel-KKT <= tol.

    fixed      -- dict(eta=..., omega=...): constant steps, every attempt accepted, no
                  restarts; runs exactly ``stop_after`` attempts.
    schedule   -- dict(attempts=[(eta, accepted), ...], checks=[(restart, to_avg), ...])
    stop_after -- stop after this many attempts (status "stopped").
    start      -- (x, y) of the ORIGINAL LP to start from instead of the projection of 0.
    on_check   -- called as on_check(attempts, best rel_kkt) at every check; returning
                  True stops the solve (status "stopped"), e.g. at a wall-clock cap.
    """
    opts = opts or PDLPOptions()
    slp, Dr, Dc = rescale(lp, opts.ruiz_iters, opts.pock_chambolle)
    K, KT = slp.K, slp.K.T.tocsr()
    c, q, l, u = slp.c, slp.q, slp.l, slp.u
    y_lo = slp.dual_lower()

    if start is None:
        x = np.clip(np.zeros(slp.n), l, u)
        y = np.maximum(np.zeros(slp.m), y_lo)
    else:
        x = np.clip(np.asarray(start[0], np.float64) / Dc, l, u)
        y = np.maximum(np.asarray(start[1], np.float64) / Dr, y_lo)
    Kx = K @ x
    KTy = KT @ y
    absmax = np.abs(K.data).max() if K.nnz else 1.0
    eta = 1.0 / absmax
    cn, qn = np.linalg.norm(c), np.linalg.norm(q)
    omega = cn / qn if (cn > 1e-10 and qn > 1e-10) else 1.0
    if fixed is not None:
        eta, omega = float(fixed["eta"]), float(fixed["omega"])

    k = 0
    accepted = 0
    restarts = 0
    since_restart = 0
    xa, ya = x.copy(), y.copy()
    xsum = np.zeros(slp.n)
    ysum = np.zeros(slp.m)
    wsum = 0.0
    kkt0, _ = _kkt_omega(slp, Dr, Dc, lp, x, y, omega)
    kkt_prev = kkt0
    attempt_log, check_log = [], []
    sched_a = schedule["attempts"] if schedule else None
    sched_c = schedule["checks"] if schedule else None
    n_check = 0
    status = "iteration_limit"
    final = None

    while True:
        for _ in range(opts.check_every):
            if k >= max_attempts or (stop_after is not None and k >= stop_after):
                break
            if sched_a is not None:
                eta = float(sched_a[k][0])
            tau, sigma = eta / omega, eta * omega
            xn = np.clip(x - tau * (c - KTy), l, u)
            Kxn = K @ xn
            yn = np.maximum(y + sigma * (q - 2.0 * Kxn + Kx), y_lo)
            k += 1
            ok_own, eta_max, eta_next = step_size_update(eta, omega, xn - x, yn - y, Kxn - Kx, k, opts)
            ok = ok_own
            if fixed is not None:
                ok, eta_next = True, eta
            if sched_a is not None:
                ok = bool(sched_a[k - 1][1])
            if record:
                attempt_log.append((eta, omega, int(ok), eta_max, eta_next, int(ok_own)))
            if ok:
                xsum += eta * xn
                ysum += eta * yn
                wsum += eta
                x, y, Kx = xn, yn, Kxn
                KTy = KT @ y
                accepted += 1
            since_restart += 1
            eta = eta_next
        stop_now = k >= max_attempts or (stop_after is not None and k >= stop_after)
        if fixed is not None or (stop_now and k % opts.check_every != 0):
            if stop_now:
                status = "stopped"
                break
            continue
        if wsum > 0:
            xbar, ybar = xsum / wsum, ysum / wsum
        else:
            xbar, ybar = x, y
        kc_cur, res_cur = _kkt_omega(slp, Dr, Dc, lp, x, y, omega)
        kc_avg, res_avg = _kkt_omega(slp, Dr, Dc, lp, xbar, ybar, omega)
        entry = dict(attempts=k, kkt_cur=kc_cur, kkt_avg=kc_avg, rel_cur=res_cur.rel_kkt,
                     rel_avg=res_avg.rel_kkt, omega=omega)
        best_avg = res_avg.rel_kkt < res_cur.rel_kkt
        if on_check is not None and on_check(k, min(res_cur.rel_kkt, res_avg.rel_kkt)) and \
                min(res_cur.rel_kkt, res_avg.rel_kkt) > tol:
            final = (xbar, ybar, res_avg) if best_avg else (x, y, res_cur)
            status = "stopped"
            check_log.append(entry)
            break
        if min(res_cur.rel_kkt, res_avg.rel_kkt) <= tol:
            final = (xbar, ybar, res_avg) if best_avg else (x, y, res_cur)
            status = "optimal"
            entry.update(restart=False, to_avg=False)
            check_log.append(entry)
            break
        if opts.eps_infeasible > 0 and fixed is None:
            infeasible = None
            for xc_, yc_ in ((x, y), (xbar, ybar)):
                rc = ray_check(lp, Dc * (xc_ - xa), Dr * (yc_ - ya))
                if rc.primal_infeasible(opts.eps_infeasible):
                    infeasible = "primal_infeasible"
                elif rc.dual_infeasible(opts.eps_infeasible):
                    infeasible = "dual_infeasible"
                if infeasible:
                    entry.update(ray=rc)
                    break
            if infeasible:
                status = infeasible
                entry.update(restart=False, to_avg=False)
                check_log.append(entry)
                break
        restart, to_avg, kc = restart_decision(kc_cur, kc_avg, wsum > 0, kkt0, kkt_prev, since_restart, k,
                                               opts)
        entry.update(restart_own=restart, to_avg_own=to_avg)
        if sched_c is not None:
            restart, to_avg = bool(sched_c[n_check][0]), bool(sched_c[n_check][1])
            kc = kc_avg if to_avg else kc_cur
        entry.update(restart=restart, to_avg=to_avg)
        kkt_prev = kc
        if restart:
            xc, yc = (xbar, ybar) if to_avg else (x, y)
            omega = primal_weight_update(omega, float(np.linalg.norm(xc - xa)), float(np.linalg.norm(yc - ya)),
                                         opts.omega_smoothing)
            x, y = xc.copy(), yc.copy()
            Kx, KTy = K @ x, KT @ y
            xa, ya = x.copy(), y.copy()
            xsum[:] = 0.0
            ysum[:] = 0.0
            wsum = 0.0
            since_restart = 0
            restarts += 1
            kkt0, _ = _kkt_omega(slp, Dr, Dc, lp, x, y, omega)
            kkt_prev = kkt0
        entry["omega_after"] = omega
        check_log.append(entry)
        n_check += 1
        if stop_now:
            status = "iteration_limit" if k >= max_attempts else "stopped"
            break

    if final is None:
        final = (x, y, kkt(lp, Dc * x, Dr * y))
    xs, ys, res = final
    xb, yb = (xsum / wsum, ysum / wsum) if wsum > 0 else (x, y)
    return PDHGResult(x=Dc * xs, y=Dr * ys, x_scaled=xs, y_scaled=ys, status=status, attempts=k,
                      accepted=accepted, restarts=restarts, rel_kkt=res.rel_kkt, primal_obj=res.primal_obj,
                      dual_obj=res.dual_obj, eta=eta, omega=omega, Dr=Dr, Dc=Dc,
                      attempt_log=attempt_log, check_log=check_log, x_cur=Dc * x, y_cur=Dr * y,
                      x_avg=Dc * xb, y_avg=Dr * yb)
