"""A randomly initialised MLP policy for RL rollouts (the action generator of
the rollout loop, vuda_rollout_run).

The paper's MLP-based RL runs a small policy network on the same GPU as the
physics and the rendering, with hidden sizes 256 and 4096 (Sec. 6.4); no
trained weights are needed to reproduce its cost.  Here the observation of
an environment is its rendered frame pooled to 16 x 16 cells per camera
(mean view depth / 4 and mean luminance per cell, one pass of the library's
vuda_observe kernel over the frame), so that inference(k + 1) depends on
render(k) as in the paper's rollout loop (Sec. 3.1), and the action is one
force per body, bounded by tanh.

    obs [E, 2 * 256 * cams] -> Linear(H) -> ReLU -> Linear(H) -> ReLU
                            -> Linear(3 N) -> tanh * max_force  -> force [3, E N]

The three layers are dense contractions: bf16 GEMMs with FP32 accumulation
on the tensor cores (cuBLAS through torch; the weights drawn in FP32 and
rounded once), the output taken back to FP32 for tanh.  The same inputs give
the same forces, so a rollout's result does not depend on how the two
groups of trajectories are scheduled.
"""
from __future__ import annotations

import numpy as np


class MLPPolicy:
    """Policy of one group of environments (all with the same body count, the
    same number of cameras and one camera size)."""

    POOL = 16   # pooled cells per image side

    def __init__(self, env, scene, hidden: int, seed: int = 0, max_force: float = 2.0, device: str = "cuda"):
        import torch
        self.env = env   # the group's batch: its frames are observed by vuda_observe
        n = np.diff(scene.body_off)
        if len(n) == 0 or (n != n[0]).any():
            raise ValueError("the policy needs the same body count in every environment")
        cams = np.diff(scene.cam_off)
        if (cams != cams[0]).any():
            raise ValueError("the policy needs the same camera count in every environment")
        W, H = int(scene.cam_w[0]), int(scene.cam_h[0])
        if (scene.cam_w != W).any() or (scene.cam_h != H).any() or W % self.POOL or H % self.POOL:
            raise ValueError("cameras must share one size, a multiple of %d" % self.POOL)
        self.E, self.N, self.cams, self.W, self.H = scene.num_envs, int(n[0]), int(cams[0]), W, H
        self.max_force = float(max_force)
        g = torch.Generator().manual_seed(seed)
        din = 2 * self.POOL * self.POOL * self.cams

        def layer(i, o):
            # default-style uniform initialisation, drawn on the host from a fixed seed
            b = 1.0 / np.sqrt(i)
            w = (torch.rand((o, i), generator=g) * 2 - 1) * b
            bias = (torch.rand(o, generator=g) * 2 - 1) * b
            return w.to(device, torch.bfloat16), bias.to(device, torch.bfloat16)

        self.layers = [layer(din, hidden), layer(hidden, hidden), layer(hidden, 3 * self.N)]
        self.obs = torch.empty((self.E, din), dtype=torch.float32, device=device)

    def observe(self, frame):
        """Observation [E, 2 * 256 * cams] of a frame (dict of rgb [P, 3] u8 and
        depth [P] f32 device tensors): per environment the 16 x 16 cell means
        of depth / 4 of its cameras, then those of luminance."""
        import torch
        self.env.observe(frame, self.POOL, 0.25, self.obs, stream=torch.cuda.current_stream())
        return self.obs

    def capture(self, frames, force, stream):
        """Capture act() for each frame of a ring as a CUDA graph on `stream`
        (the tensors are fixed: the ring's frames and the force array), so
        that a rollout's callback is one graph launch instead of a dozen
        kernel launches from Python."""
        import torch
        self._graphs = []
        with torch.cuda.stream(stream):
            for fr in frames:        # warm-up outside capture (allocator, cuBLAS workspace)
                self.act(fr, force)
        stream.synchronize()
        for fr in frames:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                self.act(fr, force)
            self._graphs.append(g)
        return self

    def act_captured(self, slot: int, stream):
        """Replay the captured act() of frame `slot` on `stream`."""
        import torch
        with torch.cuda.stream(stream):
            self._graphs[slot].replay()

    def act(self, frame, force):
        """Writes the forces of every body ([3, E N], in place) from a frame."""
        import torch
        x = self.observe(frame).to(torch.bfloat16)
        (w0, b0), (w1, b1), (w2, b2) = self.layers
        x = torch.relu(torch.addmm(b0, x, w0.t()))
        x = torch.relu(torch.addmm(b1, x, w1.t()))
        a = torch.tanh(torch.addmm(b2, x, w2.t()).float()) * self.max_force      # [E, 3 N]
        force.copy_(a.view(self.E * self.N, 3).t())
