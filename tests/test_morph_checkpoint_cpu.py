"""Checkpoint and resume of the morphing loop's optimizer state (offsets, Adam moments and step
counts, loss history), on the CPU with a stand-in loss: a run interrupted and resumed from its
checkpoint follows the uninterrupted run's trajectory bit for bit."""
import torch

from paper_2407_11272_b300.morph import load_checkpoint, optimize


def _problem():
    g = torch.Generator().manual_seed(0)
    target = torch.randn(64, 3, generator=g, dtype=torch.float32)

    def loss_of(off):
        return ((off - target) ** 2).sum() + 0.01 * (off ** 4).sum()

    off = torch.zeros(64, 3, requires_grad=True)
    return loss_of, off, torch.optim.Adam([off], lr=1e-2)


def test_resumed_run_equals_uninterrupted_run(tmp_path):
    loss_of, off_a, opt_a = _problem()
    losses_a, ran_a = optimize(loss_of, off_a, opt_a, 12)
    assert ran_a == 12 and len(losses_a) == 12

    ck = str(tmp_path / "morph.ckpt")
    loss_of, off_b, opt_b = _problem()
    optimize(loss_of, off_b, opt_b, 5, checkpoint=ck, every=2)  # "interrupted" after 5 steps
    loss_of, off_c, opt_c = _problem()  # a fresh process: new offsets and optimizer
    losses_c, ran_c = optimize(loss_of, off_c, opt_c, 12, checkpoint=ck, every=2, resume=True)
    assert ran_c == 7
    assert losses_c == losses_a
    assert torch.equal(off_c.detach(), off_a.detach())
    sa, sc = opt_a.state_dict()["state"][0], opt_c.state_dict()["state"][0]
    assert torch.equal(sa["exp_avg"], sc["exp_avg"]) and torch.equal(sa["exp_avg_sq"], sc["exp_avg_sq"])
    assert float(sa["step"]) == float(sc["step"]) == 12.0


def test_periodic_checkpoint_holds_the_state_after_its_step(tmp_path):
    ck = str(tmp_path / "morph.ckpt")
    loss_of, off, opt = _problem()
    optimize(loss_of, off, opt, 4, checkpoint=ck, every=2)
    loss_of, off2, opt2 = _problem()
    step, losses = load_checkpoint(ck, off2, opt2)
    assert step == 4 and len(losses) == 4
    assert torch.equal(off2.detach(), off.detach())
    # resuming a finished run does nothing more
    loss_of, off3, opt3 = _problem()
    _, ran = optimize(loss_of, off3, opt3, 4, checkpoint=ck, resume=True)
    assert ran == 0 and torch.equal(off3.detach(), off.detach())
