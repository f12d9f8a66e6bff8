"""Device/host ray buffers for calling the library from PyTorch.

Marshalling only: uploads seeded workloads.Rays to CUDA tensors (SoA, FP32,
16-byte aligned as the C ABI requires) and allocates output buffers.
"""
from __future__ import annotations

import numpy as np
import torch


class DeviceRays:
    """Entrance rays (x, y, dx, dy, dz) and wavelengths on the GPU."""

    def __init__(self, rays, device="cuda"):
        arrs = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
                for a in rays.arrays()]
        self.inp = arrs[:5]
        self.lam = arrs[5]
        self.n = len(rays)


class DeviceOut:
    """Exit rays (x, y, dx, dy, dz, I) and flags on the GPU."""

    def __init__(self, n, device="cuda"):
        self.f = [torch.empty(n, dtype=torch.float32, device=device) for _ in range(6)]
        self.flags = torch.empty(n, dtype=torch.uint8, device=device)
        self.n = n

    @property
    def out(self):
        return self.f + [self.flags]

    def numpy(self):
        """(out[n, 6] float32, flags[n] uint8) on the host."""
        o = torch.stack(self.f, dim=1).cpu().numpy()
        return o, self.flags.cpu().numpy()


class HostRays:
    """Host copies of entrance rays and outputs (for the *_host calls), pinned
    by default.  The six input arrays are rows of one (6, n) block and so are
    the six float outputs: the library then moves each chunk of a direction
    in one strided copy."""

    def __init__(self, rays, pin=True):
        n = len(rays)
        blk = torch.from_numpy(np.ascontiguousarray(np.stack([np.asarray(a, np.float32) for a in rays.arrays()])))
        if pin:
            blk = blk.pin_memory()
        self.inp = [blk[q] for q in range(6)]
        oblk = torch.empty((6, n), dtype=torch.float32, pin_memory=pin)
        self.out = [oblk[q] for q in range(6)]
        self.flags = torch.empty(n, dtype=torch.uint8, pin_memory=pin)
        self.n = n


class PathsOut:
    """Compacted per-path outputs of lt_trace_paths on the GPU: n_paths
    segments of `capacity` entries, plus one counter per path."""

    def __init__(self, n_paths, capacity, device="cuda"):
        m = n_paths * capacity
        self.f = [torch.empty(m, dtype=torch.float32, device=device) for _ in range(6)]
        self.flags = torch.empty(m, dtype=torch.uint8, device=device)
        self.ray_index = torch.empty(m, dtype=torch.int32, device=device)
        self.valid_count = torch.zeros(n_paths, dtype=torch.int32, device=device)
        self.n_paths, self.capacity = n_paths, capacity

    def counts(self):
        return self.valid_count.cpu().numpy().astype(np.int64)

    def path(self, p):
        """(ray_index[k], out[k, 6], flags[k]) of the entries path p wrote."""
        k = min(int(self.valid_count[p].item()), self.capacity)
        lo = p * self.capacity
        out = torch.stack([t[lo:lo + k] for t in self.f], dim=1).cpu().numpy()
        idx = self.ray_index[lo:lo + k].cpu().numpy().view(np.uint32)
        return idx, out, self.flags[lo:lo + k].cpu().numpy()
