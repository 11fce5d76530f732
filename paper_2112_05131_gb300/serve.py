"""Serving novel views of resident scenes with continuous batching over plx_render_tiles.

A trained Plenoxel grid renders a view directly (Sec. 3, no network to evaluate), so a
server keeps scenes resident in HBM and turns image requests into tiles of 16x16 pixels.
Each scheduler iteration takes tiles first-come first-served from the requests that have
arrived, up to a ray budget, uploads the tile list and launches one plx_render_tiles
over all scenes; when a request's last tile has rendered, its image is copied back to
pinned host memory on a second stream, so copies overlap the next launches.  Latency is
measured from a request's arrival to the moment its image is in host memory.

Admission is by device memory: each request is charged the device bytes of its image
while it is active (from admission until its image is back in host memory), and a
request waits in the pending queue, in arrival order, until its charge fits the
server's byte budget (by default the device's free memory at start-up, less a margin)
and a camera slot is free.  Requests admitted while others are on the GPU join the
next launch, so their work overlaps on the device.

Everything on the GPU runs in libplenoxel; this module only schedules: it fills tile
records (numpy), issues copies and launches, and polls CUDA events.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np
import torch

from .grid import MAX_TILE_SCENES, TILE_DTYPE, TILE_H, TILE_W, Grid, RenderOpts, render_tiles


@dataclass
class Request:
    rid: int
    scene: int
    cam: np.ndarray          # float32 [18]: c2w 3x4, fx, fy, cx, cy, W, H
    W: int
    H: int
    arrival: float = 0.0     # seconds on the server clock


@dataclass
class Done:
    rid: int
    arrival: float
    finished: float
    pixels: int
    image: Optional[np.ndarray] = None
    admitted: float = 0.0    # when the request left the pending queue

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def admission_wait(self) -> float:
        return self.admitted - self.arrival


@dataclass
class _Active:
    req: Request
    image: torch.Tensor          # device [H, W, 3]
    slot: int                    # camera slot
    x0: np.ndarray
    y0: np.ndarray
    charge: int                  # device bytes held until the image is back on the host
    admitted: float
    next: int = 0                # next tile to launch
    launched_all_in: int = -1    # launch id that holds the last tile


def tile_origins(W: int, H: int) -> Tuple[np.ndarray, np.ndarray]:
    """Top-left corners of the 16x16 tiles covering a W x H image, row-major."""
    ty, tx = np.meshgrid(np.arange(0, H, TILE_H, dtype=np.int32), np.arange(0, W, TILE_W, dtype=np.int32),
                         indexing="ij")
    return tx.reshape(-1), ty.reshape(-1)


def request_device_bytes(W: int, H: int) -> int:
    """Device bytes a request holds while active: its FP32 RGB image, rounded up to the caching
    allocator's 512-byte granularity."""
    return (W * H * 3 * 4 + 511) // 512 * 512


def default_memory_budget(device="cuda", margin: float = 0.1) -> int:
    """The device's free memory now, less `margin` of it (kept for the allocator and other work)."""
    free, _ = torch.cuda.mem_get_info(torch.device(device))
    return int(free * (1.0 - margin))


def scene_device_bytes(R: int, M: int, form: int = 1) -> int:
    """Device bytes of a render-only grid: index volume, rows, occupancy masks (cells and 8^3-cell blocks)
    and the rest of the workspace (an upper bound)."""
    row = 64 if form == 1 else 128
    return 4 * R ** 3 + row * M + R ** 3 // 8 + R ** 3 // 4096 + M // 8 + 4 * M + 8192


class TileServer:
    """Continuous batching of image requests over up to 8 resident scenes of one SH form."""

    def __init__(self, grids: Sequence[Grid], opts: RenderOpts = RenderOpts(), max_rays_per_launch: int = 1 << 18,
                 max_inflight: int = 2, max_active: int = 64, keep_images: bool = False, device="cuda",
                 mem_budget: Optional[int] = None):
        if not 1 <= len(grids) <= MAX_TILE_SCENES:
            raise ValueError(f"1..{MAX_TILE_SCENES} scenes")
        self.grids = list(grids)
        # device bytes that active requests may hold at once, and what they hold now
        self.mem_budget = int(mem_budget) if mem_budget is not None else default_memory_budget(device)
        self.mem_in_use = 0
        self.mem_peak = 0
        self.clock_now = 0.0
        self.opts = opts
        self.dev = torch.device(device)
        self.max_tiles = max(1, max_rays_per_launch // (TILE_W * TILE_H))
        self.max_inflight = max_inflight
        self.max_active = max_active
        self.keep_images = keep_images
        self.render_stream = torch.cuda.Stream(self.dev)
        self.copy_stream = torch.cuda.Stream(self.dev)
        # camera slots: one per active request
        self.cams_host = torch.empty((max_active, 18), dtype=torch.float32).pin_memory()
        self.cams_dev = torch.zeros((max_active, 18), dtype=torch.float32, device=self.dev)
        self.free_slots = list(range(max_active))
        # tile list buffers: one per launch in flight
        nbytes = self.max_tiles * TILE_DTYPE.itemsize
        self.tiles_host = [torch.empty(nbytes, dtype=torch.uint8).pin_memory() for _ in range(max_inflight)]
        self.tiles_dev = [torch.empty(nbytes, dtype=torch.uint8, device=self.dev) for _ in range(max_inflight)]
        self.free_tile_bufs = list(range(max_inflight))
        self.pending: collections.deque = collections.deque()   # arrived, not yet active
        self.active: collections.deque = collections.deque()    # with tiles left to launch
        self.inflight: collections.deque = collections.deque()  # (launch id, event, tile buffer, finished requests)
        self.copying: List[Tuple[torch.cuda.Event, _Active, torch.Tensor]] = []
        self.done: List[Done] = []
        self.launch_id = 0
        self.launches = 0
        self._origins: Dict[Tuple[int, int], Tuple[np.ndarray, np.ndarray]] = {}
        self._pinned: Dict[Tuple[int, int], List[torch.Tensor]] = collections.defaultdict(list)

    # ------------------------------------------------------------------ requests
    def submit(self, req: Request):
        if not 0 <= req.scene < len(self.grids):
            raise ValueError(f"request {req.rid}: no scene {req.scene}")
        if request_device_bytes(req.W, req.H) > self.mem_budget:
            raise ValueError(f"request {req.rid}: its {req.W}x{req.H} image needs more device memory than the "
                             f"server's whole budget ({self.mem_budget} bytes)")
        self.pending.append(req)

    def _activate(self):
        # first come, first served: the head of the queue waits for memory, and nothing overtakes it
        while self.pending and self.free_slots and len(self.active) + len(self.copying) < self.max_active:
            req = self.pending[0]
            charge = request_device_bytes(req.W, req.H)
            if self.mem_in_use + charge > self.mem_budget:
                break
            self.pending.popleft()
            self.mem_in_use += charge
            self.mem_peak = max(self.mem_peak, self.mem_in_use)
            slot = self.free_slots.pop()
            self.cams_host[slot] = torch.from_numpy(np.asarray(req.cam, np.float32))
            with torch.cuda.stream(self.render_stream):
                self.cams_dev[slot].copy_(self.cams_host[slot], non_blocking=True)
                image = torch.empty((req.H, req.W, 3), dtype=torch.float32, device=self.dev)
            key = (req.W, req.H)
            if key not in self._origins:
                self._origins[key] = tile_origins(req.W, req.H)
            x0, y0 = self._origins[key]
            self.active.append(_Active(req, image, slot, x0, y0, charge, self.clock_now))

    # ------------------------------------------------------------------ launches
    def _launch(self):
        if not self.active or not self.free_tile_bufs:
            return False
        buf = self.free_tile_bufs.pop()
        host = self.tiles_host[buf].numpy().view(TILE_DTYPE)
        n = 0
        finished = []
        for a in self.active:
            if n == self.max_tiles:
                break
            k = min(len(a.x0) - a.next, self.max_tiles - n)
            rec = host[n:n + k]
            rec["scene"] = a.req.scene
            rec["camera"] = a.slot
            rec["x0"] = a.x0[a.next:a.next + k]
            rec["y0"] = a.y0[a.next:a.next + k]
            rec["W"] = a.req.W
            rec["H"] = a.req.H
            rec["d_rgb"] = a.image.data_ptr()
            a.next += k
            n += k
            if a.next == len(a.x0):
                finished.append(a)
        while self.active and self.active[0].next == len(self.active[0].x0):
            self.active.popleft()
        stream = self.render_stream
        with torch.cuda.stream(stream):
            self.tiles_dev[buf][: n * TILE_DTYPE.itemsize].copy_(self.tiles_host[buf][: n * TILE_DTYPE.itemsize],
                                                                  non_blocking=True)
            render_tiles(self.grids, self.cams_dev, self.tiles_dev[buf], n, self.opts, stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.inflight.append((self.launch_id, ev, buf, finished))
        self.launch_id += 1
        self.launches += 1
        return True

    def _pinned_image(self, W: int, H: int) -> torch.Tensor:
        pool = self._pinned[(W, H)]
        return pool.pop() if pool else torch.empty((H, W, 3), dtype=torch.float32).pin_memory()

    def _poll(self, now: float):
        # launches that completed: free their tile buffer, start copies of finished requests
        while self.inflight and self.inflight[0][1].query():
            _, ev, buf, finished = self.inflight.popleft()
            self.free_tile_bufs.append(buf)
            for a in finished:
                host = self._pinned_image(a.req.W, a.req.H)
                self.copy_stream.wait_event(ev)
                with torch.cuda.stream(self.copy_stream):
                    host.copy_(a.image, non_blocking=True)
                    cev = torch.cuda.Event()
                    cev.record(self.copy_stream)
                a.image.record_stream(self.copy_stream)
                self.copying.append((cev, a, host))
        still = []
        for cev, a, host in self.copying:
            if cev.query():
                img = host.numpy().copy() if self.keep_images else None
                self._pinned[(a.req.W, a.req.H)].append(host)
                self.free_slots.append(a.slot)
                self.mem_in_use -= a.charge  # the image is released once its copy has completed
                self.done.append(Done(a.req.rid, a.req.arrival, now, a.req.W * a.req.H, img, a.admitted))
            else:
                still.append((cev, a, host))
        self.copying = still

    def idle(self) -> bool:
        return not (self.pending or self.active or self.inflight or self.copying)

    def step(self, now: float):
        """One scheduler iteration: poll completions, activate arrived requests, launch while there is room."""
        self.clock_now = now
        self._poll(now)
        self._activate()
        while len(self.inflight) < self.max_inflight and self.active:
            if not self._launch():
                break

    # ------------------------------------------------------------------ traces
    def run(self, requests: Sequence[Request], clock=time.perf_counter) -> List[Done]:
        """Serve requests whose `arrival` times are offsets from now; returns them as completed."""
        order = sorted(requests, key=lambda r: r.arrival)
        t0 = clock()
        i = 0
        self.done = []
        while i < len(order) or not self.idle():
            now = clock() - t0
            while i < len(order) and order[i].arrival <= now:
                self.submit(order[i])
                i += 1
            self.step(now)
            if self.idle() and i < len(order):
                wait = order[i].arrival - (clock() - t0)
                if wait > 2e-4:
                    time.sleep(wait - 1e-4)
        torch.cuda.synchronize(self.dev)
        return self.done


def requests_from(mix) -> List[Request]:
    """Request objects from synth.serving_requests tuples (scene, cam, W, H, arrival)."""
    return [Request(i, int(sc), cam, int(W), int(H), float(t)) for i, (sc, cam, W, H, t) in enumerate(mix)]


def latency_stats(done: Sequence[Done], wall: float) -> dict:
    lat = np.array([d.latency for d in done]) * 1e3
    wait = np.array([d.admission_wait for d in done]) * 1e3
    px = sum(d.pixels for d in done)
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "admission_wait_p50_ms": float(np.percentile(wait, 50)),
            "admission_wait_p99_ms": float(np.percentile(wait, 99)), "Mrays_per_s": px / wall / 1e6, "wall_s": wall}
