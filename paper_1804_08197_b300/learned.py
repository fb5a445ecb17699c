"""Learned reconstruction driver: training pairs from the renderer, training
and fallback-guarded inference of the residual U-Net.

Every step runs in libsg.so kernels; this module only sequences C-ABI calls
and passes device pointers (crops are pointer offsets into full images, no
copies). A pair is the plain full-rate render of a pose (W x H per eye,
step s) and the reduced render of the same pose at half resolution and twice
the step (W/2 x H/2, step 2s, at the level of detail of the full-resolution
image); the network maps the reduced render to the full-rate one. The full-rate render
is also the fallback and the yardstick: a frame whose PSNR against it falls below
the threshold is replaced by it. A learned frame (reduced render, network,
and when judged the full-rate render, the stereo PSNR and the fallback) is
one sg_render_learned call, all on the device.
"""
import numpy as np

from . import sg


class Learned:
    def __init__(self, vol, width, height, step=0.5, tau=1.0, max_batch=16, crop=64, seed=1, device="cuda",
                 slot_full=200, slot_half=201, tau_half=None):
        import torch
        self.torch = torch
        self.vol = vol
        self.W, self.H = width, height
        self.w, self.h = width // 2, height // 2
        assert self.h % 4 == 0 and self.w % 4 == 0
        self.step, self.tau = step, tau
        # the reduced render's pixel error bound: tau / 2 keeps the level of
        # detail of the full-resolution image (its pixels are twice as large)
        self.tau_half = 0.5 * tau if tau_half is None else tau_half
        self.crop = crop
        self.slot_full, self.slot_half = slot_full, slot_half
        self.net = sg.sg_unet_create(max(max_batch, 2), max(self.h, crop), max(self.w, crop), seed)
        dev = torch.device(device)
        f32 = torch.float32
        self.full = [torch.empty((self.H, self.W, 4), dtype=f32, device=dev) for _ in range(2)]
        self.half = [torch.empty((self.h, self.w, 4), dtype=f32, device=dev) for _ in range(2)]
        self.recon = [torch.empty((self.H, self.W, 4), dtype=f32, device=dev) for _ in range(2)]
        self.crop_out = torch.empty((max_batch, 2 * crop, 2 * crop, 4), dtype=f32, device=dev)
        self.loss = torch.zeros(1, dtype=f32, device=dev)
        self.psnr_buf = torch.zeros(2, dtype=f32, device=dev)
        # per judged frame: PSNR of eye 0, eye 1, the stereo pair; fallback flag
        self.max_frames = 256
        self.psnr_frames = torch.zeros((self.max_frames, 3), dtype=f32, device=dev)
        self.fell_back = torch.zeros(self.max_frames, dtype=torch.int32, device=dev)
        self.rng = np.random.default_rng(seed)
        # launch shapes (sg_render_config dicts) for full- and half-rate renders;
        # None keeps the volume's own
        self.cfg_full = self.cfg_half = None

    def close(self):
        sg.sg_unet_destroy(self.net)

    # ------------------------------------------------------------------ rendering
    def pose_full(self, views, projs, t=0):
        return sg.make_pose(views, projs, self.W, self.H, pixel_error=self.tau, t=t, slot=self.slot_full)

    def pose_half(self, views, projs, t=0):
        return sg.make_pose(views, projs, self.w, self.h, pixel_error=self.tau_half, t=t, slot=self.slot_half)

    def render_full(self, views, projs, outs=None, stream=None):
        p = self.pose_full(views, projs)
        sg.sg_select_lod(self.vol, p, stream=stream)
        if self.cfg_full is not None:
            sg.sg_set_render_config(self.vol, **self.cfg_full)
        sg.sg_render(self.vol, p, sg.render_params(step=self.step), outs or self.full, stream=stream)

    def render_half(self, views, projs, stream=None):
        p = self.pose_half(views, projs)
        sg.sg_select_lod(self.vol, p, stream=stream)
        if self.cfg_half is not None:
            sg.sg_set_render_config(self.vol, **self.cfg_half)
        sg.sg_render(self.vol, p, sg.render_params(step=2 * self.step), self.half, stream=stream)

    def tune(self, views, projs, stream=None):
        """Autotunes the launch shape of the full- and the half-rate render on
        one pose of the current volume (outputs overwritten)."""
        p = self.pose_full(views, projs)
        sg.sg_select_lod(self.vol, p, stream=stream)
        self.cfg_full, _ = sg.sg_autotune_render(self.vol, [p], sg.render_params(step=self.step), self.full,
                                                 reps=2, stream=stream)
        p = self.pose_half(views, projs)
        sg.sg_select_lod(self.vol, p, stream=stream)
        self.cfg_half, _ = sg.sg_autotune_render(self.vol, [p], sg.render_params(step=2 * self.step), self.half,
                                                 reps=2, stream=stream)

    # ------------------------------------------------------------------ training
    def _crops(self, n):
        """n random crops over the two eyes of the current pair: (in_ptrs, target_ptrs)."""
        c, f = self.crop, 4  # 4 floats per pixel
        ins, tgts = [], []
        for _ in range(n):
            e = int(self.rng.integers(0, 2))
            y = int(self.rng.integers(0, self.h - c + 1)) // 2 * 2
            x = int(self.rng.integers(0, self.w - c + 1)) // 2 * 2
            ins.append(self.half[e].data_ptr() + (y * self.w + x) * f * 4)
            tgts.append(self.full[e].data_ptr() + (2 * y * self.W + 2 * x) * f * 4)
        return ins, tgts

    def train_on_pair(self, views, projs, steps=1, batch=16, lr=5e-4, stream=None):
        """Renders one pair, then takes `steps` Adam steps on random crops of it.
        Returns the last loss (device scalar tensor)."""
        self.render_full(views, projs, stream=stream)
        self.render_half(views, projs, stream=stream)
        c = self.crop
        outs = [self.crop_out[i].data_ptr() for i in range(batch)]
        for _ in range(steps):
            ins, tgts = self._crops(batch)
            sg.sg_unet_forward(self.net, ins, self.w * 4, c, c, outs, 2 * c * 4, stream=stream)
            sg.sg_unet_backward(self.net, tgts, self.W * 4, outs, 2 * c * 4, loss=self.loss, stream=stream)
            sg.sg_unet_adam_step(self.net, lr, stream=stream)
        return self.loss

    # ------------------------------------------------------------------ inference
    def reconstruct(self, stream=None):
        """Both eyes of the current half-resolution render -> self.recon."""
        sg.sg_unet_forward(self.net, self.half, self.w * 4, self.h, self.w, self.recon, self.W * 4, stream=stream)

    def run_pipelined(self, poses, render_stream, net_stream):
        """Learned frames of `poses` with two in flight: the selection and
        half-rate render of frame i + 1 (render_stream) overlap the network on
        frame i (net_stream); the render and the network are bound by
        different units (instruction issue; copies and tensor cores) and share
        the SMs. Half-rate images and reconstructions are double-buffered; a
        render waits for the network to have read its buffer. Returns the
        device time from the first render to the last reconstruction (ms);
        the reconstructions stay in self.recon_pair."""
        torch = self.torch
        if not hasattr(self, "half_pair"):
            self.half_pair = [self.half, [torch.empty_like(h) for h in self.half]]
            self.recon_pair = [self.recon, [torch.empty_like(r) for r in self.recon]]
        ev = lambda: torch.cuda.Event(enable_timing=False)
        rendered, consumed = [ev(), ev()], [None, None]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(render_stream)
        net_stream.wait_event(start)
        for i, (views, projs) in enumerate(poses):
            k = i % 2
            if consumed[k] is not None:
                render_stream.wait_event(consumed[k])
            p = self.pose_half(views, projs)
            sg.sg_select_lod(self.vol, p, stream=render_stream)
            if self.cfg_half is not None:
                # one CTA per tile: a persistent grid holds every SM until its
                # queue drains and would not share them with the network
                sg.sg_set_render_config(self.vol, **dict(self.cfg_half, persistent=0))
            sg.sg_render(self.vol, p, sg.render_params(step=2 * self.step), self.half_pair[k], stream=render_stream)
            rendered[k].record(render_stream)
            net_stream.wait_event(rendered[k])
            sg.sg_unet_forward(self.net, self.half_pair[k], self.w * 4, self.h, self.w, self.recon_pair[k], self.W * 4,
                               stream=net_stream)
            consumed[k] = ev()
            consumed[k].record(net_stream)
        end.record(net_stream)
        torch.cuda.synchronize()
        return start.elapsed_time(end)

    def run_plain_pipelined(self, poses, render_stream, sel_stream, slots=(202, 203)):
        """Plain full-rate frames of `poses` with the selection of frame i + 1
        (sel_stream, its own slot of two) overlapping the render of frame i
        (render_stream); a slot is selected again only after the render that
        read it. Returns the device time from the first selection to the
        last render (ms); the images stay in self.full."""
        torch = self.torch
        ev = lambda: torch.cuda.Event(enable_timing=False)
        selected, read = [ev(), ev()], [None, None]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(render_stream)
        sel_stream.wait_event(start)
        if self.cfg_full is not None:
            sg.sg_set_render_config(self.vol, **self.cfg_full)
        for i, (views, projs) in enumerate(poses):
            k = i % 2
            p = sg.make_pose(views, projs, self.W, self.H, pixel_error=self.tau, slot=slots[k])
            if read[k] is not None:
                sel_stream.wait_event(read[k])
            sg.sg_select_lod(self.vol, p, stream=sel_stream)
            selected[k].record(sel_stream)
            render_stream.wait_event(selected[k])
            sg.sg_render(self.vol, p, sg.render_params(step=self.step), self.full, stream=render_stream)
            read[k] = ev()
            read[k].record(render_stream)
        end.record(render_stream)
        torch.cuda.synchronize()
        return start.elapsed_time(end)

    def psnr(self, a, b, out_index=0, stream=None):
        sg.sg_psnr(a, b, a.numel(), self.psnr_buf[out_index:out_index + 1], stream=stream)
        return self.psnr_buf[out_index:out_index + 1]

    def learned_params(self, judge=False, threshold_db=40.0):
        return sg.learned_params(step=self.step, pixel_error_half=self.tau_half, threshold_db=threshold_db,
                                 judge=judge, half_slot=self.slot_half, half_config=self.cfg_half,
                                 full_config=self.cfg_full)

    def frame(self, views, projs, judge=False, threshold_db=40.0, index=0, stream=None):
        """One learned stereo frame (sg_render_learned) into self.recon. Judged,
        it also renders the full-rate frame into the network's buffer and
        writes the PSNRs of the pair to psnr_frames[index] and the fallback
        flag to fell_back[index] (device; nothing waits)."""
        pose = self.pose_full(views, projs)
        prm = self.learned_params(judge, threshold_db)
        sg.sg_render_learned(self.vol, self.net, pose, prm, self.recon,
                             self.psnr_frames[index] if judge else None, self.fell_back[index:index + 1] if judge else None,
                             stream=stream)

    def evaluate(self, views, projs, index=0, stream=None):
        """Judges one pose's learned frame; returns its stereo PSNR (dB), reading
        the device value (the one host wait of this call)."""
        self.frame(views, projs, judge=True, index=index, stream=stream)
        return float(self.psnr_frames[index, 2].item())
