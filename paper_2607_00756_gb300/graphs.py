"""Maps of several specimens (one built BipContext each: uneven grids,
slice counts, f, channel counts, precisions) captured into one CUDA graph
and replayed.  The contexts are switched to capture-safe mode (no host
synchronisation inside a map; uploads only when the scans change), warmed
up once with the same arguments, then captured; a replay re-runs every
launch of every map with no host work.  Marshalling only: the launches are
the library's."""
import numpy as np
import torch

from . import capi


class GraphedMaps:
    def __init__(self, items, concurrent=True):
        """items: [(BipContext, H, scans)], each context built.  concurrent:
        each specimen's launches on a stream of its own, forked from and
        joined back to the capturing stream, so that the graph's branches
        (the specimens share no buffers) can run side by side and small
        specimens fill the GPU together; otherwise one after another."""
        self.items = [(b, H, np.asarray(sc, dtype=np.float64)) for b, H, sc in items]
        if not self.items:
            raise ValueError("no specimens")
        dev = self.items[0][1].device
        self.outs = [torch.empty(len(sc), dtype=torch.float64, device=dev) for _, _, sc in self.items]
        self.streams = [torch.cuda.Stream(device=dev) for _ in self.items] if concurrent else None
        for b, _, _ in self.items:
            capi.bip_set_capture_safe(b.ctx, True)
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            self._run()                               # allocations, uploads, kernel attributes
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.check()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._run()

    def _run(self):
        if self.streams is None:
            for (b, H, sc), o in zip(self.items, self.outs):
                b.map(H, sc, out=o)
            return
        main = torch.cuda.current_stream()
        for (b, H, sc), o, st in zip(self.items, self.outs, self.streams):
            st.wait_stream(main)                      # fork
            with torch.cuda.stream(st):
                b.map(H, sc, out=o)
        for st in self.streams:
            main.wait_stream(st)                      # join

    def replay(self):
        """Re-run every map; returns the output tensors (one per specimen)."""
        self.graph.replay()
        return self.outs

    def check(self):
        """Raise if a device-side wait of any map gave up (synchronises)."""
        for b, _, _ in self.items:
            capi.bip_check_errors(b.ctx)
