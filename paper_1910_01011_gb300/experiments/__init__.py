"""Reproductions of the paper's experiments on synthetic inputs."""
