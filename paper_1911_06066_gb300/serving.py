"""Open-loop load for the request server: Poisson arrivals of MLMC level-pair
sample requests, mixed over levels, with latency percentiles.

The arrival process is the caller's (synthetic) workload, not part of the
method: inter-arrival times are exponential with the given rate, each
request's level is drawn from ``level_mix``, sample ids count up per level,
and -- for the per-request variant -- each request gets its own 64-bit seed
and a stimulus centre uniform in a box.  Latency is measured from the
scheduled arrival time (so a late submission by this loop counts against the
server) to the time the server saw the batch finish.
"""
import time

import numpy as np

from .binding import Server, mlmc_request


def poisson_schedule(rate, n, level_mix, rng_seed=0, seed=0, per_request_seed=False,
                     stim_box=None, dim=2):
    """Arrival times [n] (s), levels, seeds, sample ids and stimulus centres."""
    rng = np.random.default_rng(rng_seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    p = np.asarray(level_mix, np.float64)
    levels = rng.choice(len(p), size=n, p=p / p.sum())
    ids = np.zeros(n, np.int64)
    nxt = np.zeros(len(p), np.int64)
    for i, l in enumerate(levels):
        ids[i] = nxt[l]
        nxt[l] += 1
    if per_request_seed:
        seeds = rng.integers(0, 2 ** 63, size=n, dtype=np.int64).astype(np.uint64)
    else:
        seeds = np.full(n, seed, np.uint64)
    stim = None
    if stim_box is not None:
        lo, hi = stim_box
        stim = np.zeros((n, 3))
        stim[:, :dim] = rng.uniform(lo, hi, size=(n, dim))
    return t, levels, seeds, ids, stim


def run_open_loop(server, schedule, eps=None, check_every=0.25, timeout=600.0):
    """Submits the schedule at its arrival times, collects every result and
    returns a report: offered rate, completed requests per second, p50/p99
    latency, queue and batch statistics, and (if eps is given) the time at
    which the running estimate's sampling error sqrt(sum V_l / N_l) first
    fell to eps / sqrt(2) -- submission stops there."""
    t_arr, levels, seeds, ids, stim = schedule
    n = len(t_arr)
    reqs = Server.requests(np.arange(n), levels, seeds, ids, stim)
    t0 = server.clock()
    sent = 0
    results = []
    t_reached = None
    last_check = 0.0
    deadline = time.monotonic() + timeout
    while True:
        now = server.clock() - t0
        k = sent
        while k < n and t_arr[k] <= now:
            k += 1
        if k > sent:
            server.submit((mlmc_request * (k - sent))(*reqs[sent:k]))
            sent = k
        results.extend(server.poll(timeout=0.0005))
        if eps is not None and t_reached is None and now - last_check >= check_every:
            last_check = now
            est = server.estimate()
            N = est["N_l"]
            if np.all(N > 1):
                stat = float(np.sqrt(np.sum(est["V_l"] / N)))
                if stat <= eps / np.sqrt(2.0):
                    t_reached = now
                    n = sent          # stop offering load
        if sent >= n and len(results) >= sent:
            break
        if time.monotonic() > deadline:
            raise TimeoutError("open-loop run did not finish in %.0f s" % timeout)
        if sent < n:
            wait = t_arr[sent] - (server.clock() - t0)
            if wait > 0.0005:
                time.sleep(min(wait, 0.002))
    lat = np.array([r["t_done"] - t0 - t_arr[r["tag"]] for r in results])
    span = max(r["t_done"] for r in results) - t0 if results else 0.0
    st = server.stats()
    est = server.estimate()
    return dict(
        offered_rate=float(len(results) / t_arr[len(results) - 1]) if results else 0.0,
        completed=len(results), seconds=span,
        throughput=len(results) / span if span > 0 else 0.0,
        p50_ms=float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
        p99_ms=float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
        max_queue=st["max_queue"], batches=st["batches"], arena_peak_bytes=st["arena_peak_bytes"],
        failed=int(sum(r["status"] != 0 for r in results)),
        time_to_eps=t_reached, N_l=est["N_l"].tolist(), V_l=est["V_l"].tolist(),
        rmse=est["rmse"], bias=est["bias"],
        stat_err=float(np.sqrt(np.sum(est["V_l"] / np.maximum(est["N_l"], 1)))),
        results=results)
