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
    """Pinned host copies of entrance rays and outputs (for the *_host calls)."""

    def __init__(self, rays, pin=True):
        self.inp = [torch.from_numpy(np.ascontiguousarray(a, np.float32)) for a in rays.arrays()]
        if pin:
            self.inp = [t.pin_memory() for t in self.inp]
        n = len(rays)
        self.out = [torch.empty(n, dtype=torch.float32, pin_memory=pin) for _ in range(6)]
        self.flags = torch.empty(n, dtype=torch.uint8, pin_memory=pin)
        self.n = n
