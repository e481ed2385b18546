"""Load increments captured as CUDA graphs.

An increment is one or more ``dmn_eval`` launches (one per DMN handle, e.g.
trees of different depth in one batch) on fixed device buffers.  The launch
sequence is captured once per state parity (state A -> B and B -> A) and then
replayed; the caller copies the next increment's inputs into ``deps`` and
``theta`` before each replay.  ``dmn_eval`` allocates nothing and does not
synchronise, so it can be captured; the handles must be created (and their
kernels configured) before capture, which ``DMN.__init__`` does.
"""
from __future__ import annotations


class IncrementGraph:
    def __init__(self, parts, dt=1.0):
        """parts: list of (dmn, n_points) evaluated one after the other."""
        import torch

        self.parts = parts
        self.dt = float(dt)
        dev = torch.device("cuda", torch.cuda.current_device())
        f64, i32 = torch.float64, torch.int32
        self.deps = [torch.zeros((n, 6), dtype=f64, device=dev) for _, n in parts]
        self.theta = [torch.full((n,), 293.0, dtype=f64, device=dev) for _, n in parts]
        self.state = [[torch.zeros((n, d.state_words), dtype=f64, device=dev) for _ in range(2)]
                      for d, n in parts]
        self.out = [torch.zeros((n, 57), dtype=f64, device=dev) for _, n in parts]
        self.status = [torch.zeros(n, dtype=i32, device=dev) for _, n in parts]
        self.iters = [torch.zeros(n, dtype=i32, device=dev) for _, n in parts]
        self.parity = 0
        self.graphs = []
        for par in range(2):
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):  # warm-up outside capture
                self._launch(par)
            torch.cuda.current_stream().wait_stream(s)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._launch(par)
            self.graphs.append(g)

    def _launch(self, par):
        for i, (d, _) in enumerate(self.parts):
            d.eval(self.deps[i], self.theta[i], self.dt, self.state[i][par],
                   self.state[i][1 - par], self.out[i], self.status[i], self.iters[i])

    def set_state(self, i, state):
        self.state[i][self.parity].copy_(state)

    def current_state(self, i):
        return self.state[i][self.parity]

    def step(self):
        """Replay one increment; the output state becomes the next input."""
        self.graphs[self.parity].replay()
        self.parity = 1 - self.parity


class WarmIncrementGraph:
    """One increment of the learned-warm-start path -- network input
    (``dmn_mlp_input``), the network's four GEMMs (``dmn_mlp_predict``) and
    the warm-started solve (``dmn_eval_warm``) -- captured as CUDA graphs.

    The path reads the states of the two previous increments and writes the
    next, so three state buffers rotate; one graph is captured per rotation
    phase.  Before each ``step`` the caller writes the increment's inputs
    into ``deps`` and ``theta``; ``out``, ``status``, ``iters`` and ``da``
    hold the results of the last replay."""

    def __init__(self, dmn, net, n, prev, cur, dt=1.0):
        """prev, cur: the states after the two previous increments."""
        import torch

        self.dmn, self.net, self.n, self.dt = dmn, net, int(n), float(dt)
        dev = torch.device("cuda", torch.cuda.current_device())
        f64, i32 = torch.float64, torch.int32
        self.deps = torch.zeros((n, 6), dtype=f64, device=dev)
        # the first launches (outside capture) run a zero load step at the
        # current temperature: one Newton iteration per point
        self.theta = cur[:, 6].clone()
        self.state = [prev.clone(), cur.clone(), torch.empty_like(cur)]
        self.xin = torch.zeros((n, net.n_in_pad), dtype=torch.bfloat16, device=dev)
        self.da = torch.zeros((n, net.n_out), dtype=torch.float32, device=dev)
        self.out = torch.zeros((n, 57), dtype=f64, device=dev)
        self.status = torch.zeros(n, dtype=i32, device=dev)
        self.iters = torch.zeros(n, dtype=i32, device=dev)
        self.phase = 0
        self.graphs = []
        for ph in range(3):
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):  # first launches outside capture (kernel set-up)
                self._launch(ph)
            torch.cuda.current_stream().wait_stream(s)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._launch(ph)
            self.graphs.append(g)
        self.set_states(prev, cur)

    def _launch(self, ph):
        prev, cur, nxt = self.state[ph], self.state[(ph + 1) % 3], self.state[(ph + 2) % 3]
        self.net.input(self.deps, self.theta, cur, prev, out=self.xin)
        self.net.predict(self.xin, out=self.da)
        self.dmn.eval_warm(self.deps, self.theta, self.dt, cur, self.da, nxt, self.out, self.status,
                           self.iters)

    def set_states(self, prev, cur):
        """States after the two previous increments (copied in)."""
        self.state[self.phase].copy_(prev)
        self.state[(self.phase + 1) % 3].copy_(cur)

    def current_state(self):
        return self.state[(self.phase + 1) % 3]

    def previous_state(self):
        return self.state[self.phase]

    def step(self):
        """Replay one increment; the new state becomes the current one."""
        self.graphs[self.phase].replay()
        self.phase = (self.phase + 1) % 3
