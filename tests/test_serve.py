"""Host-side logic of the continuously batching server, with a fake executor
(no GPU): batching, admission under the HBM cap with eviction of idle
slots, oldest-first service across geometries, one slot per geometry for
both ops without mixing them in a batch, requests that fail on the host
without blocking the others, and the latency report."""
import itertools

from paper_2510_01785_gb300.serve import Request, Server, latency_report, make_requests


class FakeExecutor:
    """A slot is busy for `work` pump calls after a launch."""

    def __init__(self, bytes_per_slot=10, work=2):
        self.bps, self.work = bytes_per_slot, work
        self.ids = itertools.count()
        self.live = {}
        self.launches = []

    def slot_bytes(self, nside, lmax, max_ch):
        return self.bps * (2 if nside >= 1024 else 1)

    def new_slot(self, nside, lmax, max_ch):
        h = {"id": next(self.ids), "nside": nside, "left": 0, "batch": [], "bytes": self.slot_bytes(nside, lmax, max_ch)}
        self.live[h["id"]] = h
        return h

    def handle_bytes(self, h):
        return h["bytes"]

    def free_slot(self, h):
        assert h["left"] == 0
        del self.live[h["id"]]

    def launch(self, h, op, batch):
        assert sum(r.nch for r in batch) <= 32 and len({(r.nside, r.op) for r in batch}) == 1
        h["left"], h["batch"] = self.work, batch
        self.launches.append((h["id"], op, [r.rid for r in batch]))

    def done(self, h):
        h["left"] -= 1
        return h["left"] <= 0

    def finish(self, h):
        return [f"out{r.rid}" for r in h["batch"]]


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-3
        return self.t


def drain(srv, limit=10000):
    for _ in range(limit):
        srv.pump()
        if not srv.pending() and not srv.busy():
            return
    raise AssertionError("server did not drain")


def test_requests_arriving_together_are_packed_into_batches():
    ex = FakeExecutor()
    srv = Server(ex, hbm_cap_bytes=100, max_channels=32, max_slots_per_key=1, clock=Clock())
    reqs = [Request(rid=i, op="map2alm", nside=64, nch=5) for i in range(20)]
    for r in reqs:
        srv.submit(r)
    drain(srv)
    assert all(r.y == f"out{r.rid}" and r.error is None for r in reqs)
    # 20 x 5 channels in batches of at most 6 requests (30 channels)
    assert len(ex.launches) == 4 and max(len(b) for _, _, b in ex.launches) == 6
    served = [rid for _, _, b in ex.launches for rid in b]
    assert served == list(range(20))  # arrival order kept


def test_late_arrivals_join_the_next_batch_while_a_batch_runs():
    ex = FakeExecutor(work=3)
    srv = Server(ex, hbm_cap_bytes=100, max_channels=32, max_slots_per_key=1, clock=Clock())
    srv.submit(Request(rid=0, op="alm2map", nside=16, nch=4))
    srv.pump()  # launches rid 0
    for i in range(1, 5):
        srv.submit(Request(rid=i, op="alm2map", nside=16, nch=4))
    drain(srv)
    assert [b for _, _, b in ex.launches] == [[0], [1, 2, 3, 4]]


def test_admission_never_exceeds_the_cap_and_evicts_idle_slots():
    ex = FakeExecutor(bytes_per_slot=10, work=2)
    srv = Server(ex, hbm_cap_bytes=25, max_channels=32, max_slots_per_key=2, clock=Clock())
    reqs = [Request(rid=i, op="map2alm" if i % 2 else "alm2map", nside=[16, 32, 64][i % 3], nch=20)
            for i in range(30)]
    for r in reqs:
        srv.submit(r)
        srv.pump()
        assert srv.bytes <= 25
    drain(srv)
    assert srv.peak_bytes <= 25
    assert all(r.y is not None for r in reqs)
    assert len(ex.live) <= 2


def test_bad_requests_fail_on_the_host_and_do_not_block_others():
    ex = FakeExecutor()
    srv = Server(ex, hbm_cap_bytes=15, max_channels=32, clock=Clock())
    bad = [Request(rid=100, op="map2alm", nside=12, nch=1), Request(rid=101, op="map2alm", nside=16, nch=40),
           Request(rid=102, op="fft", nside=16, nch=1), Request(rid=103, op="map2alm", nside=1024, nch=1)]
    good = [Request(rid=i, op="map2alm", nside=16, nch=2) for i in range(3)]
    for r in bad + good:
        srv.submit(r)
    drain(srv)
    assert all(r.error for r in bad) and "cap" in bad[3].error
    assert all(r.error is None and r.y == f"out{r.rid}" for r in good)
    rep = latency_report(bad + good)
    assert rep["errors"] == 4 and rep["served"] == 3


def test_make_requests_is_seeded_and_follows_the_mix():
    a = make_requests(7, 500.0, 2.0, {64: 0.5, 1024: 0.5})
    b = make_requests(7, 500.0, 2.0, {64: 0.5, 1024: 0.5})
    assert [(r.op, r.nside, r.nch, r.t_arrival) for r in a] == [(r.op, r.nside, r.nch, r.t_arrival) for r in b]
    assert 800 < len(a) < 1200
    assert all(1 <= r.nch <= 32 and r.lmax == 3 * r.nside - 1 for r in a)
    assert 0.4 < sum(r.op == "map2alm" for r in a) / len(a) < 0.6


def test_oldest_waiting_request_goes_first_across_geometries():
    """With memory for one slot, the geometry whose head request arrived
    first is served first, and the idle slot of the other is evicted."""
    ex = FakeExecutor(bytes_per_slot=10, work=2)
    clk = Clock()
    srv = Server(ex, hbm_cap_bytes=10, max_channels=32, max_slots_per_key=1, clock=clk)
    srv.submit(Request(rid=0, op="map2alm", nside=32, nch=4, t_arrival=0.5))
    srv.submit(Request(rid=1, op="map2alm", nside=16, nch=4, t_arrival=0.1))
    srv.submit(Request(rid=2, op="map2alm", nside=32, nch=4, t_arrival=0.6))
    drain(srv)
    assert [b for _, _, b in ex.launches] == [[1], [0, 2]]
    assert srv.peak_bytes <= 10


def test_ops_share_a_geometry_slot_but_not_a_batch():
    ex = FakeExecutor()
    srv = Server(ex, hbm_cap_bytes=100, max_channels=32, max_slots_per_key=1, clock=Clock())
    for i in range(6):
        srv.submit(Request(rid=i, op="map2alm" if i % 2 else "alm2map", nside=64, nch=3))
    drain(srv)
    slots = {h for h, _, _ in ex.launches}
    assert len(slots) == 1  # one slot for the geometry, both ops on it
    for _, op, b in ex.launches:
        assert all((rid % 2 == 1) == (op == "map2alm") for rid in b)
    assert sorted(rid for _, _, b in ex.launches for rid in b) == list(range(6))


def test_latency_report_percentiles():
    reqs = []
    for i in range(100):
        r = Request(rid=i, op="map2alm", nside=16, nch=1, t_arrival=float(i))
        r.t_done = r.t_arrival + (i + 1) * 1e-3  # latencies 1 .. 100 ms
        reqs.append(r)
    bad = Request(rid=100, op="map2alm", nside=16, nch=1)
    bad.error, bad.t_done = "rejected", 0.0
    rep = latency_report(reqs + [bad])
    assert rep["requests"] == 101 and rep["served"] == 100 and rep["errors"] == 1
    assert abs(rep["p50_ms"] - 50.5) < 1e-9 and abs(rep["p99_ms"] - 99.01) < 1e-9
    assert abs(rep["mean_ms"] - 50.5) < 1e-9


class WideExecutor(FakeExecutor):
    """Batches of up to 96 channels at Nside 2048, the default elsewhere."""

    def batch_capacity(self, nside, lmax):
        return 96 if nside == 2048 else 32

    def launch(self, h, op, batch):
        cap = self.batch_capacity(batch[0].nside, batch[0].lmax)
        assert sum(r.nch for r in batch) <= cap and len({(r.nside, r.op) for r in batch}) == 1
        h["left"], h["batch"] = self.work, batch
        self.launches.append((h["id"], op, [r.rid for r in batch]))


def test_batch_capacity_may_exceed_one_requests_limit():
    """A geometry whose slots take 96 channels packs several 32-channel
    requests into one call; requests are still limited to 32 channels."""
    ex = WideExecutor()
    srv = Server(ex, hbm_cap_bytes=100, max_channels=32, max_slots_per_key=1, clock=Clock())
    reqs = [Request(rid=i, op="alm2map", nside=2048, nch=30) for i in range(9)]
    reqs.append(Request(rid=9, op="alm2map", nside=2048, nch=33))
    for r in reqs:
        srv.submit(r)
    drain(srv)
    assert reqs[9].error is not None and "channels" in reqs[9].error
    assert all(r.y == f"out{r.rid}" for r in reqs[:9])
    assert [len(b) for _, _, b in ex.launches] == [3, 3, 3]


def test_evictions_are_counted():
    ex = FakeExecutor(bytes_per_slot=10)
    srv = Server(ex, hbm_cap_bytes=20, max_channels=32, max_slots_per_key=1, clock=Clock())
    for i, ns in enumerate([64, 128, 256, 64, 512]):
        srv.submit(Request(rid=i, op="map2alm", nside=ns, nch=4))
        drain(srv)
    # two slots fit: 256 evicts 64's (LRU), 64 evicts 128's, 512 evicts 256's
    assert srv.evictions == 3 and srv.bytes <= 20


class OverEstimating(FakeExecutor):
    """Estimates 3x the bytes a slot turns out to hold."""

    def slot_bytes(self, nside, lmax, max_ch):
        return 3 * super().slot_bytes(nside, lmax, max_ch)

    def handle_bytes(self, h):
        return h["bytes"] // 3  # what the built slot holds


def test_admission_uses_measured_slot_sizes_once_known():
    """The first slot of a geometry is admitted on the estimate; later ones
    on the size the first one measured, so an over-estimate does not keep
    evicting slots that in fact fit."""
    ex = OverEstimating(bytes_per_slot=10)
    srv = Server(ex, hbm_cap_bytes=35, max_channels=32, max_slots_per_key=1, clock=Clock())
    for i, ns in enumerate([64, 128, 256]):  # estimates 30 each: every new geometry evicts the other slot
        srv.submit(Request(rid=i, op="map2alm", nside=ns, nch=4))
        drain(srv)
    assert srv.evictions == 2 and srv.known_bytes[(64, 191)] == 10
    for i, ns in enumerate([64, 128, 256, 64, 128]):  # now known: 10 each, all three fit 35
        srv.submit(Request(rid=10 + i, op="map2alm", nside=ns, nch=4))
        drain(srv)
    assert srv.evictions == 2  # no more: re-admitting 64 and 128 fits beside 256
    assert len([s for ss in srv.slots.values() for s in ss]) == 3


def test_streamed_slots_hold_no_table():
    """The executor's plan flags per geometry (a geometry in both lists gets
    the table) and the admission estimate of a streamed slot: no table, so
    well under the table slot of the same geometry."""
    from paper_2510_01785_gb300 import _lib
    from paper_2510_01785_gb300.serve import GpuExecutor
    ex = GpuExecutor(device="cpu", lambda_table_nsides=(256,), streamed_nsides=(256, 1024))
    stream = _lib.HPX_PLAN_LAMBDA_TABLE | _lib.HPX_PLAN_TENSOR_CORES | _lib.HPX_PLAN_LAMBDA_STREAM
    assert ex._flags(1024) == stream
    assert ex._flags(256) == _lib.HPX_PLAN_LAMBDA_TABLE | _lib.HPX_PLAN_TENSOR_CORES
    assert ex._flags(64) == _lib.HPX_PLAN_LAMBDA_RECOMPUTE
    tab = GpuExecutor(device="cpu", lambda_table_nsides=(1024,)).slot_bytes(1024, 3071, 32)
    assert 0 < ex.slot_bytes(1024, 3071, 32) < tab / 3
