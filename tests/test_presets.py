"""The paper presets against the paper's tables (no GPU): TurtleBot2 and Go2
geometry and action bounds (Tables 8-9), shared sensing and episode
constants (Table 7), the training pipeline (Tables 3-5)."""
import math

from paper_2606_15846_b300 import train as TR
from paper_2606_15846_b300 import workloads as W


def test_robot_presets_tables_8_9():
    tb, go = W.TURTLEBOT2, W.GO2
    assert (tb.shape, tb.radius) == (0, 0.20)
    assert (go.shape, go.length, go.width) == (1, 0.80, 0.41)
    for r in (tb, go):
        assert (r.v_min, r.v_max) == (0.0, 0.5)
        assert math.isclose(r.w_max, math.pi / 4) and math.isclose(r.w_min, -math.pi / 4)


def test_shared_sensing_and_episode_table_7():
    wl = W.config_paper("turtlebot2", n_envs=8)
    p = wl.params
    assert (p.sensor, p.march_step, p.n_sectors) == (1, 0.03, 30)
    assert wl.max_range == 20.0 and int(wl.env_beams[0]) == 1080
    assert 1080 // p.n_sectors == 36
    assert (p.dt, p.goal_tol, p.horizon) == (0.1, 0.2, 200)
    assert (p.c_progress, p.r_goal, p.r_coll, p.reward_mode) == (2.0, 10.0, 10.0, 1)
    assert p.fov_deg == 270.0 and W.config_paper("go2", n_envs=8).params.fov_deg == 360.0
    # map sizes: 10 x 10 m and 13.5 x 13.5 m at 0.05 m
    assert wl.maps[0].shape == (200, 200)
    assert W.config_paper("go2", n_envs=8).maps[0].shape == (270, 270)
    assert len(wl.maps) == 1 and (wl.env_map == 0).all()  # one shared bitmap


def test_training_pipeline_tables_3_to_5():
    c = TR.paper_config("turtlebot2")
    assert (c.n_envs, c.batch, c.utd, c.learning_starts) == (1024, 1024, 40, 8192)
    assert (c.hidden, c.n_hidden, c.gamma, c.weight_decay) == (100, 4, 0.97, 1e-3)
    assert c.ipap and c.overlap and c.steps_per_sync == 1 and c.algo == "fastdsac"
    assert (c.policy_freq, c.reward_scale) == (2, 0.4)
    assert TR.paper_config("go2").steps_per_sync == 2
    s = TR.paper_config("turtlebot2", "fastsac")
    assert (s.algo, s.policy_freq) == ("fastsac", 1)
    assert TR.paper_config("go2", "fastsac").policy_freq == 2
    assert TR.obs_features(c) + 4 == 34
