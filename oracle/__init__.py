"""FP64 CPU oracle for the dynamic-human renderer (test infrastructure only).

A plain, slow, obviously-correct restatement of what the renderer computes,
written from the paper: volume rendering (Sec. 2.1, Eq. 2-3), the
observation-to-canonical motion field (Sec. 4, M = M_skel + M_res), inverse
linear-blend skinning (Sec. 4.2), the pose-conditioned residual MLP with its
positional encoding and truncated Hann window (Sec. 4.3), the canonical field
and the likelihood augmentation (Sec. 4.4), and the squared-error loss
(Sec. 2.1, Sec. 5.2).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA path; the two
meet only in the seeded input generator ``paper_2306_16541_gb300.synth``.

Modules:
  fk        forward kinematics -> per-bone inverse transforms G_i (Sec. 4.2)
  field     the per-point field: warp, residual, encoding, MLP (Sec. 4.2-4.4)
  render    rays, sampling, compositing, loss (Sec. 2.1, 4.4, 5.2)
  decide32  the float32 decisions that select samples (box clip, occupancy
            cell, posed occupancy bitfield), taken in the kernel's precision
  rng       SplitMix64 counter generator for stratified jitter
"""
