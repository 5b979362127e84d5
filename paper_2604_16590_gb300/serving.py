"""Request loop of the serving engine: submits requests at their arrival times
and drives engine iterations of the C-ABI server (gattn_serve_*) until every
request has finished.  Host orchestration only; all device work is the
library's ragged attention and merge-update launches."""
from __future__ import annotations

import time

import torch

from . import gattn
from .inputs import pooled_state, request_state


def run(server: gattn.Server, specs, Y=32, X=64, d=64, device="cuda", realtime=True, on_done=None, pool=None):
    """Serve `specs` (inputs.ServeRequestSpec); returns {request index: latency_s}.

    With realtime=True a request is submitted once the wall clock passes its
    arrival time (engine iterations keep running meanwhile), otherwise all
    requests are submitted up front in arrival order.  With `pool` (see
    inputs.state_pool) the initial states are views into that device buffer."""
    pending = sorted(range(len(specs)), key=lambda i: specs[i].arrival_s)
    ids = {}
    lat = {}
    t0 = time.perf_counter()
    k = 0
    while len(lat) < len(specs):
        now = time.perf_counter() - t0
        while k < len(pending) and (not realtime or specs[pending[k]].arrival_s <= now):
            i = pending[k]
            if pool is not None:
                z0 = pooled_state(specs[i], pool, Y, X, d)
            else:
                z0 = request_state(specs[i], Y, X, d, device=device)
            ids[i] = server.submit(z0)
            k += 1
        active, waiting = server.step()
        for i, rid in list(ids.items()):
            if i in lat:
                continue
            if server.done(rid):
                _, lat_s = gattn.gattn_serve_poll(server.h, rid, None)[1:]
                lat[i] = lat_s
                if on_done:
                    on_done(i, rid)
        if active == 0 and waiting == 0 and k < len(pending) and realtime:
            time.sleep(max(0.0, min(0.01, specs[pending[k]].arrival_s - (time.perf_counter() - t0))))
    return lat
