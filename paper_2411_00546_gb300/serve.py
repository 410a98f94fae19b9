"""Request loop over the continuous-batching server (ras_server_* in the C ABI).

Requests arrive at given times; the loop submits every request whose arrival
time has passed on the wall clock, advances the server by one step (admission
within the HBM budget, then one outer RASPEN iteration of every admitted
request in shared launches), and fetches finished results. The latency of a
request is its completion time minus its arrival time.
"""
import time

from . import ras


def percentile(values, q):
    """q-th percentile (0..100) by linear interpolation between order statistics."""
    v = sorted(values)
    if not v:
        return None
    x = (len(v) - 1) * q / 100.0
    lo = int(x)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (x - lo)


def run_stream(requests, hbm_budget, max_active, opts=None, stream=None, keep_results=False, graphs=False):
    """requests: list of (t_arrival_s, problem dict with host y_d), sorted by
    arrival. Returns a dict with per-request latency (s), status, stats, the
    steps taken, the largest admitted set and (optionally) the results.
    graphs: CUDA graphs in the server's workspaces."""
    s = ras.ras_server_create(hbm_budget, max_active, opts, stream)
    ras.ras_server_use_graphs(s, graphs)
    try:
        order = sorted(range(len(requests)), key=lambda i: requests[i][0])
        rid_of, arrival, done_at, status, stats, results = {}, {}, {}, {}, {}, {}
        nxt = 0
        steps = 0
        peak_active = 0
        peak_bytes = 0
        t0 = time.perf_counter()
        while len(done_at) < len(requests):
            now = time.perf_counter() - t0
            while nxt < len(order) and requests[order[nxt]][0] <= now:
                i = order[nxt]
                rid_of[ras.ras_server_submit(s, requests[i][1])] = i
                arrival[i] = requests[i][0]
                nxt += 1
            pend, act, _ = ras.ras_server_counts(s)
            if pend == 0 and act == 0:
                if nxt < len(order):
                    wait = requests[order[nxt]][0] - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(wait)
                    continue
                break
            act, _ = ras.ras_server_step(s)
            steps += 1
            peak_active = max(peak_active, act)
            peak_bytes = max(peak_bytes, ras.ras_server_device_bytes(s))
            t_now = time.perf_counter() - t0
            for rid in ras.ras_server_finished_ids(s):
                rc, y, p, st = ras.ras_server_fetch(s, rid)
                i = rid_of.pop(rid)
                done_at[i] = t_now
                status[i] = rc
                stats[i] = st.as_dict()
                if keep_results:
                    results[i] = (y, p)
        lat = {i: done_at[i] - arrival[i] for i in done_at}
        return {"latency_s": lat, "status": status, "stats": stats, "steps": steps,
                "peak_active": peak_active, "peak_device_bytes": peak_bytes,
                "wall_s": max(done_at.values()) if done_at else 0.0,
                "first_arrival_s": min(arrival.values()) if arrival else 0.0, "results": results}
    finally:
        ras.ras_server_destroy(s)
