"""ADMM for  min <C, X>  s.t.  diag(X) = 1,  X PSD, as a stream of projection
requests for the request server.

The three-step scheme of Sec. 5 ("ADMM for SDP", Eq. exp:admm-three-step)
with A(X) = diag(X), A*(y) = Diag(y), b = 1, so that A A* = I:
    y_{k+1} = b / sigma - diag(X_k / sigma + S_k - C)
    S_{k+1} = Pi( C - Diag(y_{k+1}) - X_k / sigma )
    X_{k+1} = X_k + sigma (S_{k+1} + Diag(y_{k+1}) - C)
The projection Pi is one server request per iteration; the y- and X-updates
are the solver's own work on its device tensors (they are not part of the
projection).  Progress is measured with the surrogate KKT residual of Sec. 5
(primal infeasibility, dual infeasibility, relative gap).

`Solve` holds one solve's iterates; `run_serving` interleaves many solves
whose arrivals are Poisson and whose iterations are closed-loop (the next
request is issued a random think time after the previous one completes);
`solve` runs one solve to a tolerance with the warm-start schedule of Sec. 5
(low-precision projections until the surrogate first drops below 1e-2, then
high-precision ones).
"""
import math
import time

import numpy as np


class Solve:
    """One ADMM solve on torch tensors (any device).

    C: symmetric (n, n) float32 tensor, shared read-only between solves.
    The projection input V and output S are (n, n) row-major tensors; for a
    symmetric matrix the row/column-major distinction does not matter, and
    the projection writes both triangles.
    """

    def __init__(self, C, sigma, iters, stream=None):
        import torch
        self.torch = torch
        self.C = C
        self.n = C.shape[0]
        self.sigma = float(sigma)
        self.iters = int(iters)
        self.k = 0
        self.stream = stream
        self.X = torch.zeros_like(C)
        self.S = torch.zeros_like(C)
        self.V = torch.empty_like(C)
        self.y = torch.zeros(self.n, dtype=C.dtype, device=C.device)
        self.ready = torch.cuda.Event() if C.is_cuda else None

    def _ctx(self):
        if self.stream is not None:
            return self.torch.cuda.stream(self.stream)
        import contextlib
        return contextlib.nullcontext()

    def make_input(self):
        """y-update and the projection input V = C - Diag(y) - X / sigma."""
        s = self.sigma
        with self._ctx():
            dX, dS, dC = self.X.diagonal(), self.S.diagonal(), self.C.diagonal()
            self.y.copy_(1.0 / s - (dX / s + dS - dC))
            self.torch.add(self.C, self.X, alpha=-1.0 / s, out=self.V)
            self.V.diagonal().sub_(self.y)
            if self.ready is not None:
                self.ready.record(self.stream if self.stream is not None else self.torch.cuda.current_stream())
        return self.V

    def finish_iteration(self):
        """X-update with S = Pi(V) in place; returns True when the solve is done."""
        s = self.sigma
        with self._ctx():
            self.X.add_(self.S, alpha=s)
            self.X.add_(self.C, alpha=-s)
            self.X.diagonal().add_(self.y, alpha=s)
        self.k += 1
        return self.k >= self.iters

    def surrogate(self):
        """max(primal infeasibility, dual infeasibility, relative gap) (Sec. 5)."""
        torch = self.torch
        with self._ctx():
            X, S, C, y = self.X.double(), self.S.double(), self.C.double(), self.y.double()
            b_norm = math.sqrt(self.n)
            pinf = float(torch.linalg.vector_norm(X.diagonal() - 1.0)) / (1.0 + b_norm)
            R = S - C
            R.diagonal().add_(y)
            dinf = float(torch.linalg.matrix_norm(R)) / (1.0 + float(torch.linalg.matrix_norm(C)))
            pobj = float((C * X).sum())
            dobj = float(y.sum())
            gap = abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))
        return max(pinf, dinf, gap), dict(pinf=pinf, dinf=dinf, gap=gap, pobj=pobj, dobj=dobj)


def run_serving(server, graphs, precision="fp16", solve_rate=8.0, arrival_seconds=2.5, iters=50,
                think_ms=0.5, seed=0, sigma_range=(0.5, 2.0), max_solves=None):
    """Interleaved ADMM solves as a request stream against a psd_server.

    graphs: {n: C} device float32 tensors (one Laplacian per size class).
    Solves arrive as a Poisson process of rate `solve_rate` per second during
    `arrival_seconds`, each on a size class drawn uniformly, with its own
    sigma drawn log-uniformly from sigma_range; each runs `iters` iterations,
    issuing the next request an Exp(think_ms) time after the previous one
    completes.  Returns per-request records and per-solve summaries.
    """
    import torch
    from . import binding as b
    rng = np.random.default_rng(seed)
    sizes = sorted(graphs)
    arrivals = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / solve_rate)
        if t > arrival_seconds or (max_solves is not None and len(arrivals) >= max_solves):
            break
        n = sizes[rng.integers(len(sizes))]
        sig = math.exp(rng.uniform(math.log(sigma_range[0]), math.log(sigma_range[1])))
        arrivals.append((t, n, sig))
    stream = torch.cuda.Stream()
    records, solves_done = [], []
    active = []  # dicts: solve, state ("think" | "wait"), t_next, ticket
    t0 = time.perf_counter()
    nxt = 0
    while nxt < len(arrivals) or active:
        now = time.perf_counter() - t0
        while nxt < len(arrivals) and arrivals[nxt][0] <= now:
            _, n, sig = arrivals[nxt]
            active.append(dict(solve=Solve(graphs[n], sig, iters, stream), state="think", t_next=now,
                               ticket=None, t_start=now))
            nxt += 1
        still = []
        for a in active:
            sv = a["solve"]
            if a["state"] == "think" and now >= a["t_next"]:
                V = sv.make_input()
                a["ticket"] = b.psd_server_submit(server, sv.n, V, sv.n, sv.S, sv.n, precision, ready=sv.ready)
                a["state"] = "wait"
            if a["state"] == "wait":
                done, info, lat = b.psd_server_poll(server, a["ticket"])
                if done:
                    records.append(dict(n=sv.n, latency_ms=lat, status=info["status"],
                                        lambda_bound=info["lambda_bound"]))
                    finished = sv.finish_iteration()
                    if finished:
                        stream.synchronize()
                        eta, parts = sv.surrogate()
                        solves_done.append(dict(n=sv.n, sigma=sv.sigma, iters=sv.k, eta=eta,
                                                seconds=now - a["t_start"], **parts))
                        continue
                    a["state"] = "think"
                    a["t_next"] = now + rng.exponential(think_ms * 1e-3)
            still.append(a)
        active = still
        if active and all(a["state"] == "wait" for a in active) and nxt >= len(arrivals):
            time.sleep(50e-6)
    stream.synchronize()
    wall = time.perf_counter() - t0
    return dict(records=records, solves=solves_done, wall_s=wall, arrivals=len(arrivals))


def summarize(result):
    """Per size class and overall: count, p50/p99 latency (ms), projections/s and TFLOP/s
    (22 n^3 per half-precision projection: 22 products of n^3 multiply-adds' worth)."""
    recs = result["records"]
    wall = result["wall_s"]
    out = {"wall_s": wall, "solves": len(result["solves"]), "requests": len(recs)}
    classes = {}
    for n in sorted({r["n"] for r in recs}):
        lat = np.array([r["latency_ms"] for r in recs if r["n"] == n])
        classes[str(n)] = {"count": int(lat.size), "p50_ms": float(np.percentile(lat, 50)),
                           "p99_ms": float(np.percentile(lat, 99))}
    lat = np.array([r["latency_ms"] for r in recs]) if recs else np.zeros(1)
    flops = sum(22.0 * r["n"] ** 3 for r in recs)
    out.update(per_class=classes, p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
               projections_per_s=len(recs) / wall if wall > 0 else 0.0,
               tflops=flops / wall / 1e12 if wall > 0 else 0.0,
               bad_status=sum(1 for r in recs if r["status"] != 0))
    if result["solves"]:
        sizes = sorted({s["n"] for s in result["solves"]})
        out["eta_median_by_n"] = {str(n): float(np.median([s["eta"] for s in result["solves"] if s["n"] == n]))
                                  for n in sizes}
        # the surrogate's parts (Sec. 5): primal and dual infeasibility, relative gap
        out["eta_parts_median_by_n"] = {
            str(n): {k: float(np.median([s[k] for s in result["solves"] if s["n"] == n]))
                     for k in ("pinf", "dinf", "gap")} for n in sizes}
    return out


def solve(C, project, sigma=1.0, max_iters=5000, eta_switch=1e-2, eta_tol=1e-4, check_every=10,
          low="mixed", high="fp32"):
    """The ADMM solver of Sec. 5 with its warm-start schedule: iterate with the
    `low` precision projection until the surrogate KKT residual (primal and
    dual infeasibility, relative gap) first drops below eta_switch, then with
    `high` until it drops below eta_tol or max_iters is reached.

    project(V, S, precision) writes Pi(V) into S (both (n, n) tensors on C's
    device; on a GPU, e.g. a psd_project call).  The surrogate is evaluated
    every `check_every` iterations.  Returns dict(X, S, y, iters, switch_iter,
    history=[(iteration, precision, eta)]).
    """
    sv = Solve(C, sigma, max_iters)
    prec = low
    switch_iter = None
    history = []
    for k in range(1, max_iters + 1):
        V = sv.make_input()
        project(V, sv.S, prec)
        sv.finish_iteration()
        if k % check_every == 0 or k == max_iters:
            eta, _ = sv.surrogate()
            history.append((k, prec, eta))
            if prec == low and eta < eta_switch:
                prec, switch_iter = high, k
            elif prec == high and eta < eta_tol:
                break
    return dict(X=sv.X, S=sv.S, y=sv.y, iters=k, switch_iter=switch_iter, history=history)
